// diffusion.cu -- the diffusion step of the advection-diffusion scheme
// (arXiv 2103.02388, Sec. 2.2, Eq. finite-dimensional Galerkin approximation
// and Eq. linear system; Algorithm 1 line 5, and the two fractional steps of
// the Strang splitting, Algorithm 2):
//
//   (M + tau theta kappa A) c^{n+1} = (M - tau (1 - theta) kappa A) c_hat
//                                     + tau M q,        c = c_bnd on the boundary,
//
// with the P1 / P2 mass matrix M and stiffness matrix A of the refined mesh,
// solved by Jacobi-preconditioned conjugate gradients (the system matrix is
// symmetric positive definite, Sec. 2.2).
//
// Matrix-free operator.  Every macro is an affine image of the reference
// Kuhn simplex, and its micro simplices are the Kuhn simplices (one per axis
// permutation sigma) of the lattice cells, so all micro simplices of a macro
// with the same sigma are translates of one another: their element
// matrices are equal.  The host computes, per macro, the mass matrix (the
// same for every sigma, since all micro simplices have the same volume) and
// one stiffness matrix per sigma.
//
// Node-centred stencil in the macro interiors.  A node strictly inside a
// macro lies only in micro simplices of that macro, and those of one
// orientation are translates of one another, so its row of the assembled
// matrix depends only on its class (its lattice coordinates mod P: vertex or
// one of the edge-midpoint classes) and the macro: the host sums the element
// matrices into per-class, per-macro weights at fixed lattice offsets
// (StencilShape: 65 offsets for the 3D P2 vertex class, 19 or 27 for its edge
// classes), and k_stencil applies them, one warp per 32 interior nodes of
// one class (from host-built lists in storage order), each lane one node,
// every neighbour read directly from the storage layout.  No atomics; each
// node's row sum has a fixed order.
//
// Face nodes shared by two or more macros take explicit rows, assembled on
// the host from every micro simplex holding them (k_face_rows, one warp per
// row); rows of Dirichlet nodes are never formed, since the solver never
// reads them.
//
// A blended mesh, whose simplices each have their own matrices, takes every
// cell through a cell pass instead: two lattice cells whose indices have the
// same parity in every axis share no node, so each of the 2^d parities
// (colours) has its own accumulator vector in the storage layout; within one
// colour every slot has at most one writing thread, which stores its cell's
// sum over the cell's simplices, and all colours run in one launch.  The
// accumulators are tiled by 32 slots: accumulator (slot, colour) sits at
// ((slot / 32) 2^d + colour) 32 + slot % 32.  Every accumulator that some
// cell of its colour covers is rewritten on every application, and the
// others stay zero from the set-up.  A fold then adds, for every node, its
// storage copies in ascending slot order and each copy's colours in
// ascending order, and writes the sum to every copy.
//
// The summation order is fixed everywhere, so results are bitwise equal run
// to run.  The solver's vectors are in the storage layout (the copies of an
// interface node hold the same value); dot products count the owner copy of
// each unknown.  Each dot product is completed inside the kernel that forms
// its partials (the last block to finish sums them in a fixed order), which
// also sets the done flag once the residual or the iteration budget is
// reached; every later kernel of the batch then returns at once, and the host
// reads the scalars once per kCheckEvery iterations.
//
// Dirichlet conditions: boundary unknowns keep c_bnd; CG runs on the
// interior unknowns (search directions are zero on the boundary).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "elm_internal.h"

namespace elm {
namespace {

constexpr int kDiffThreads = 128;
constexpr int kRedThreads = 256;
// Grid of the vector kernels and reductions: about 4 values per thread, at
// most kRedMaxBlocks blocks (the partials of one reduction).
constexpr int kRedMaxBlocks = 8192;
inline int red_blocks(int64_t n) {
  const int64_t b = (n + 4 * kRedThreads - 1) / (4 * kRedThreads);
  return int(b < 1 ? 1 : (b > kRedMaxBlocks ? kRedMaxBlocks : b));
}

__host__ __device__ constexpr int n_local(int d, int p) { return p == 2 ? (d + 1) * (d + 2) / 2 : d + 1; }
__host__ __device__ constexpr int n_perm(int d) { return d == 3 ? 6 : 2; }

// The axis permutations of a cell in lexicographic order (3D: 012, 021, 102,
// 120, 201, 210; 2D: 01, 10).
__host__ __device__ inline void perm_of(int d, int k, int* s) {
  if (d == 2) {
    s[0] = k;
    s[1] = 1 - k;
    return;
  }
  const int t[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  s[0] = t[k][0];
  s[1] = t[k][1];
  s[2] = t[k][2];
}

// ---------------------------------------------------------------------------
// Host: element matrices.
// ---------------------------------------------------------------------------

// A polynomial term c * prod lam_k^e_k of the barycentric coordinates.
struct Term {
  double c;
  int e[4];
};

double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }

// int over a simplex of unit volume of prod lam_k^e_k: d! e_0! .. e_d! / (d + |e|)!.
double monomial_unit(int d, const int* e) {
  double num = fact(d);
  int tot = 0;
  for (int k = 0; k <= d; ++k) {
    num *= fact(e[k]);
    tot += e[k];
  }
  return num / fact(d + tot);
}

// Local basis in the order vertices 0..d, then edges (a, b), a < b,
// lexicographic (P2); vertices only (P1).
std::vector<std::vector<Term>> basis_terms(int d, int p) {
  std::vector<std::vector<Term>> B;
  for (int v = 0; v <= d; ++v) {
    std::vector<Term> t;
    Term sq{2.0, {0, 0, 0, 0}}, li{-1.0, {0, 0, 0, 0}}, one{1.0, {0, 0, 0, 0}};
    sq.e[v] = 2;
    li.e[v] = 1;
    one.e[v] = 1;
    if (p == 2) {
      t.push_back(sq);
      t.push_back(li);
    } else {
      t.push_back(one);
    }
    B.push_back(t);
  }
  if (p == 2)
    for (int a = 0; a <= d; ++a)
      for (int b = a + 1; b <= d; ++b) {
        Term t{4.0, {0, 0, 0, 0}};
        t.e[a] = 1;
        t.e[b] = 1;
        B.push_back({t});
      }
  return B;
}

// d phi_i / d lam_k = a[i][k] + sum_m b[i][k][m] lam_m (linear for P1 and P2).
void basis_derivatives(int d, int p, std::vector<double>& a, std::vector<double>& b) {
  const int nb = n_local(d, p), D1 = d + 1;
  a.assign(nb * D1, 0.0);
  b.assign(nb * D1 * D1, 0.0);
  for (int v = 0; v <= d; ++v) {
    if (p == 2) {  // 2 lam_v^2 - lam_v
      a[v * D1 + v] = -1.0;
      b[(v * D1 + v) * D1 + v] = 4.0;
    } else {  // lam_v
      a[v * D1 + v] = 1.0;
    }
  }
  if (p == 2) {
    int i = d + 1;
    for (int s = 0; s <= d; ++s)
      for (int t = s + 1; t <= d; ++t, ++i) {  // 4 lam_s lam_t
        b[(i * D1 + s) * D1 + t] = 4.0;
        b[(i * D1 + t) * D1 + s] = 4.0;
      }
  }
}

// Element tables of one macro: mass (nb x nb) and one stiffness matrix per
// permutation ([n_perm, nb, nb]), FP64.
void element_tables(int d, int p, int N, const MacroGeo& g, double* Mout, double* Aout) {
  const int nb = n_local(d, p), D1 = d + 1;
  // reference mass on unit volume
  const auto B = basis_terms(d, p);
  std::vector<double> Mref(nb * nb);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double s = 0.0;
      for (const Term& ti : B[i])
        for (const Term& tj : B[j]) {
          int e[4];
          for (int k = 0; k < 4; ++k) e[k] = ti.e[k] + tj.e[k];
          s += ti.c * tj.c * monomial_unit(d, e);
        }
      Mref[i * nb + j] = s;
    }
  std::vector<double> da, db;
  basis_derivatives(d, p, da, db);
  // K[i][j][k][l] = int_unit (dphi_i/dlam_k)(dphi_j/dlam_l), with
  // int lam_m = 1/(d+1), int lam_m lam_n = (1 + delta_mn)/((d+1)(d+2)).
  std::vector<double> K(nb * nb * D1 * D1);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j)
      for (int k = 0; k < D1; ++k)
        for (int l = 0; l < D1; ++l) {
          const double ai = da[i * D1 + k], aj = da[j * D1 + l];
          double sbi = 0.0, sbj = 0.0, bb = 0.0;
          for (int m = 0; m < D1; ++m) {
            sbi += db[(i * D1 + k) * D1 + m];
            sbj += db[(j * D1 + l) * D1 + m];
            for (int n = 0; n < D1; ++n)
              bb += db[(i * D1 + k) * D1 + m] * db[(j * D1 + l) * D1 + n] * (m == n ? 2.0 : 1.0);
          }
          K[((i * nb + j) * D1 + k) * D1 + l] =
              ai * aj + (ai * sbj + aj * sbi) / double(D1) + bb / double(D1 * (D1 + 1));
        }
  for (int sg = 0; sg < n_perm(d); ++sg) {
    int s[3];
    perm_of(d, sg, s);
    // vertices of the cell-0 Kuhn simplex: w_0 = 0, w_k = w_{k-1} + e_{s_{k-1}}
    double V[4][3] = {};
    int w[3] = {0, 0, 0};
    for (int k = 0; k <= d; ++k) {
      if (k > 0) w[s[k - 1]] += 1;
      for (int r = 0; r < d; ++r) {
        double x = g.v0[r];
        for (int c = 0; c < d; ++c) x += g.J[r * 3 + c] * (double(w[c]) / double(N));
        V[k][r] = x;
      }
    }
    // barycentric gradients: rows of E^{-1}, E = [V1 - V0 | ... ]
    double E[9], Ei[9];
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) E[r * d + c] = V[c + 1][r] - V[0][r];
    double det;
    if (d == 2) {
      det = E[0] * E[3] - E[1] * E[2];
      Ei[0] = E[3] / det;
      Ei[1] = -E[1] / det;
      Ei[2] = -E[2] / det;
      Ei[3] = E[0] / det;
    } else {
      const double c00 = E[4] * E[8] - E[5] * E[7], c01 = E[5] * E[6] - E[3] * E[8], c02 = E[3] * E[7] - E[4] * E[6];
      det = E[0] * c00 + E[1] * c01 + E[2] * c02;
      Ei[0] = c00 / det;
      Ei[1] = (E[2] * E[7] - E[1] * E[8]) / det;
      Ei[2] = (E[1] * E[5] - E[2] * E[4]) / det;
      Ei[3] = c01 / det;
      Ei[4] = (E[0] * E[8] - E[2] * E[6]) / det;
      Ei[5] = (E[2] * E[3] - E[0] * E[5]) / det;
      Ei[6] = c02 / det;
      Ei[7] = (E[1] * E[6] - E[0] * E[7]) / det;
      Ei[8] = (E[0] * E[4] - E[1] * E[3]) / det;
    }
    const double vol = std::fabs(det) / (d == 2 ? 2.0 : 6.0);
    double G[4][3] = {};
    for (int k = 1; k <= d; ++k)
      for (int r = 0; r < d; ++r) {
        G[k][r] = Ei[(k - 1) * d + r];
        G[0][r] -= G[k][r];
      }
    if (sg == 0)
      for (int i = 0; i < nb * nb; ++i) Mout[i] = vol * Mref[i];
    double* A = Aout + size_t(sg) * nb * nb;
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double a = 0.0;
        for (int k = 0; k < D1; ++k)
          for (int l = 0; l < D1; ++l) {
            double gg = 0.0;
            for (int r = 0; r < d; ++r) gg += G[k][r] * G[l][r];
            a += gg * K[((i * nb + j) * D1 + k) * D1 + l];
          }
        A[i * nb + j] = vol * a;
      }
  }
}

// Element tables of a mesh blended onto an annulus (2D; elm_mesh_set_annulus):
// one mass and one stiffness matrix per micro simplex, [n_macros][T2(N)
// cells][2 orientations][2][nb * nb], zero for simplices outside the macro.
// With the polar sector map the Jacobian determinant is the constant
// Delta / sin(Delta), so the mass is the affine one times it; the stiffness is
// int grad_x phi_i^T G grad_x phi_j with the metric
//   G = DPhi^{-1} DPhi^{-T} |det DPhi| = (Delta / sin Delta) (w w^T / Delta^2 + p p^T),
// w = e_{k+1} - e_k, p = (1 - lam) e_k + lam e_{k+1}, lam the sector parameter
// of the point, integrated with a 5 x 5 collapsed Gauss-Legendre rule.
void blended_element_tables(const elm_mesh_s* me, std::vector<double>& out) {
  const int d = 2, p = me->order, nb = n_local(d, p), N = me->N, D1 = 3;
  const int64_t ncell = int64_t(N) * (N + 1) / 2;
  out.assign(size_t(me->n_macros) * ncell * 2 * 2 * nb * nb, 0.0);
  const auto B = basis_terms(d, p);
  std::vector<double> Mref(nb * nb);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double s = 0.0;
      for (const Term& ti : B[i])
        for (const Term& tj : B[j]) {
          int e[4];
          for (int k = 0; k < 4; ++k) e[k] = ti.e[k] + tj.e[k];
          s += ti.c * tj.c * monomial_unit(d, e);
        }
      Mref[i * nb + j] = s;
    }
  std::vector<double> da, db;
  basis_derivatives(d, p, da, db);
  const double delta = me->blend.delta, jac = delta / std::sin(delta);
  // 5-point Gauss-Legendre on [-1, 1]
  const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831, 0.9061798459386640};
  const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889, 0.4786286704993665,
                        0.2369268850561891};
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const MacroGeo& g = me->geo[m];
    // the macro's sector: from its centroid (every macro spans one sector)
    double cx = g.v0[0] + (2.0 * g.J[0] + g.J[1]) / 3.0, cy = g.v0[1] + (2.0 * g.J[3] + g.J[4]) / 3.0;
    const double tt = (std::atan2(cy, cx) - me->blend.theta0) / delta;
    int k = int(std::floor(tt)) % me->blend.nsec;
    if (k < 0) k += me->blend.nsec;
    const double tk = me->blend.theta0 + k * delta;
    const double ek[2] = {std::cos(tk), std::sin(tk)}, ek1[2] = {std::cos(tk + delta), std::sin(tk + delta)};
    const double w[2] = {ek1[0] - ek[0], ek1[1] - ek[1]};
    for (int c0 = 0; c0 < N; ++c0)
      for (int c1 = 0; c1 <= c0; ++c1)
        for (int sg = 0; sg < 2; ++sg) {
          int s[2];
          perm_of(2, sg, s);
          const int c[2] = {c0, c1};
          if (c[s[0]] == c[s[1]] && s[0] > s[1]) continue;  // outside the macro
          double V[3][2];
          int wl[2] = {c0, c1};
          for (int v = 0; v <= 2; ++v) {
            if (v > 0) wl[s[v - 1]] += 1;
            for (int r = 0; r < 2; ++r)
              V[v][r] = g.v0[r] + g.J[r * 3 + 0] * (double(wl[0]) / N) + g.J[r * 3 + 1] * (double(wl[1]) / N);
          }
          const double E00 = V[1][0] - V[0][0], E01 = V[2][0] - V[0][0], E10 = V[1][1] - V[0][1],
                       E11 = V[2][1] - V[0][1];
          const double det = E00 * E11 - E01 * E10, area = 0.5 * std::fabs(det);
          // barycentric gradients: rows of E^{-1} for lam_1, lam_2
          double G[3][2];
          G[1][0] = E11 / det;
          G[1][1] = -E01 / det;
          G[2][0] = -E10 / det;
          G[2][1] = E00 / det;
          G[0][0] = -G[1][0] - G[2][0];
          G[0][1] = -G[1][1] - G[2][1];
          double* Me = out.data() + ((size_t(m) * ncell + size_t(c0) * (c0 + 1) / 2 + c1) * 2 + sg) * 2 * nb * nb;
          double* Ae = Me + nb * nb;
          for (int i = 0; i < nb * nb; ++i) Me[i] = area * Mref[i] * jac;
          for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) {
              const double u = 0.5 * (gx[a] + 1.0), v = 0.5 * (gx[b] + 1.0);
              const double lam[3] = {1.0 - u, u * (1.0 - v), u * v};
              const double W = 0.25 * gw[a] * gw[b] * u * 2.0 * area;
              const double x = lam[0] * V[0][0] + lam[1] * V[1][0] + lam[2] * V[2][0];
              const double y = lam[0] * V[0][1] + lam[1] * V[1][1] + lam[2] * V[2][1];
              const double ck = ek[0] * y - ek[1] * x, ck1 = ek1[0] * y - ek1[1] * x;
              const double sl = ck / (ck - ck1);
              const double pp[2] = {(1.0 - sl) * ek[0] + sl * ek1[0], (1.0 - sl) * ek[1] + sl * ek1[1]};
              double Gm[2][2];
              for (int r = 0; r < 2; ++r)
                for (int q = 0; q < 2; ++q) Gm[r][q] = jac * (w[r] * w[q] / (delta * delta) + pp[r] * pp[q]);
              double gr[6][2];
              for (int i = 0; i < nb; ++i) {
                gr[i][0] = gr[i][1] = 0.0;
                for (int kk = 0; kk < D1; ++kk) {
                  double dk = da[i * D1 + kk];
                  for (int mm = 0; mm < D1; ++mm) dk += db[(i * D1 + kk) * D1 + mm] * lam[mm];
                  gr[i][0] += dk * G[kk][0];
                  gr[i][1] += dk * G[kk][1];
                }
              }
              for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j)
                  Ae[i * nb + j] += W * (gr[i][0] * (Gm[0][0] * gr[j][0] + Gm[0][1] * gr[j][1]) +
                                         gr[i][1] * (Gm[1][0] * gr[j][0] + Gm[1][1] * gr[j][1]));
            }
        }
  }
}

// ---------------------------------------------------------------------------
// Device: the operator y += scale (M + alpha A) x.
// ---------------------------------------------------------------------------

// CG scalars on the device.  done: the residual or the iteration budget was
// reached; iters: iterations completed; arrived: blocks of the current grid
// that have written their partial (the last one completes the reduction).
struct Scalars {
  double rz, rz_new, pq, rr, bb, alpha, beta, stop_rr;
  int done, iters, budget;
  unsigned arrived;
};

// Updates the CG scalars from reduced sums a (and b):
// what = 1: p.q -> alpha; 2: (r.z, r.r) -> beta, one iteration done, and the
// done flag once |r|^2 <= stop_rr (or it is not finite) or the budget is spent.
__device__ __forceinline__ void cg_scalars_update(int what, double a, double b, Scalars* sc) {
  if (what == 1) {
    sc->pq = a;
    sc->alpha = a != 0.0 ? sc->rz / a : 0.0;
  } else {
    sc->rz_new = a;
    sc->rr = b;
    sc->beta = sc->rz != 0.0 ? a / sc->rz : 0.0;
    sc->rz = a;
    sc->iters += 1;
    if (b <= sc->stop_rr || !isfinite(b) || sc->iters >= sc->budget) sc->done = 1;
  }
}

// What an operator pass does with its result v at a node.
enum OpMode {
  kOpAccum = 0,  // y += v
  kOpCg = 1,     // y = v (0 on the Dirichlet boundary), and a partial of p.y (x = p)
  kOpDiag = 2    // y += the diagonal entry (x unused)
};

struct OpArgs {
  const void* tables;       // blended meshes: per-simplex mass and stiffness
  const int4* chunks;       // cell pass: (macro, first cell, count, colour) per block
  const int4* cellv;        // cells (c0, c1, c2) of all colours, macro by macro
  int npm;                  // storage nodes per macro
  int N;                    // 2^L
  const Scalars* sc;        // CG scalars: the kernels return once sc->done is set (null: always run)
};

__device__ __forceinline__ int tri2d(int k) { return k * (k + 1) / 2; }
__device__ __forceinline__ int tri3d(int k) { return k * (k + 1) * (k + 2) / 6; }

// Axis sigma_k of permutation sg (the order of perm_of), as a constant
// expression for the unrolled simplex loop of k_apply.
__host__ __device__ constexpr int perm_axis(int d, int sg, int k) {
  return d == 2 ? (k == 0 ? sg : 1 - sg)
                : (sg == 0 ? (k == 0 ? 0 : k == 1 ? 1 : 2)
                   : sg == 1 ? (k == 0 ? 0 : k == 1 ? 2 : 1)
                   : sg == 2 ? (k == 0 ? 1 : k == 1 ? 0 : 2)
                   : sg == 3 ? (k == 0 ? 1 : k == 1 ? 2 : 0)
                   : sg == 4 ? (k == 0 ? 2 : k == 1 ? 0 : 1)
                             : (k == 0 ? 2 : k == 1 ? 1 : 0));
}
// Node lattice offset along axis r of vertex k of the Kuhn simplex sg of a
// cell (P node points per cell edge): P times the number of the first k
// sorted axes equal to r.
__host__ __device__ constexpr int vtx_off(int d, int sg, int k, int r, int P) {
  return P * ((k > 0 && perm_axis(d, sg, 0) == r) + (k > 1 && perm_axis(d, sg, 1) == r) +
              (k > 2 && perm_axis(d, sg, 2) == r));
}
// Local node j of the simplex (vertices, then edges (u, v), u < v,
// lexicographic), as an index of the cell's (P + 1)^d node box.
__host__ __device__ constexpr int edge_u(int d, int j) {
  return d == 3 ? (j == 4 || j == 5 || j == 6 ? 0 : j == 7 || j == 8 ? 1 : 2) : (j == 3 || j == 4 ? 0 : 1);
}
__host__ __device__ constexpr int edge_v(int d, int j) {
  return d == 3 ? (j == 4 ? 1 : j == 5 || j == 7 ? 2 : 3) : (j == 3 ? 1 : 2);
}
__host__ __device__ constexpr int node_off(int d, int sg, int j, int r, int P) {
  return j <= d ? vtx_off(d, sg, j, r, P)
                : (vtx_off(d, sg, edge_u(d, j), r, P) + vtx_off(d, sg, edge_v(d, j), r, P)) / 2;
}
template <int D, int P>
__host__ __device__ constexpr int local_index(int sg, int j) {
  return D == 3 ? (node_off(D, sg, j, 0, P) * (P + 1) + node_off(D, sg, j, 1, P)) * (P + 1) + node_off(D, sg, j, 2, P)
                : node_off(D, sg, j, 0, P) * (P + 1) + node_off(D, sg, j, 1, P);
}

// Node-centred stencil of the assembled operator inside a macro.  A node q
// strictly inside a macro's reference simplex lies only in micro simplices of
// that macro, and the simplices of one orientation sigma are translates of
// one another, so row q of the assembled matrix depends only on the class of
// q (q mod P per axis: the vertex class and, for P2, the edge-midpoint
// classes) and on the macro: entry (q, q + o) is the sum, over the simplices
// holding q as their local node i, of the element entries (i, j) with node j
// at offset o.  StencilShape lists, per class, the offsets o that occur
// (lexicographic order) and the index of o = 0; the weights are per macro
// (stencil_weights).  3D P2: 65 offsets for the vertex class, 19 or 27 for
// the edge classes; P1: 15 (3D), 7 (2D).
template <int D, int P>
struct StencilShape {
  static constexpr int NCLS = P == 2 ? (1 << D) : 1;
  static constexpr int MAXE = D == 3 ? (2 * P + 1) * (2 * P + 1) * (2 * P + 1) : (2 * P + 1) * (2 * P + 1);
  int n[NCLS];             // offsets of class k
  int start[NCLS + 1];     // first entry of class k in the per-macro weight table
  int centre[NCLS];        // entry of o = 0 within class k
  int off[NCLS][MAXE][3];  // offsets (axis 0 = q0, the slowest axis of the packed index)
  __host__ __device__ constexpr StencilShape() : n{}, start{}, centre{}, off{} {
    for (int sg = 0; sg < n_perm(D); ++sg)
      for (int i = 0; i < n_local(D, P); ++i) {
        const int k = class_of_node(sg, i);
        for (int j = 0; j < n_local(D, P); ++j) {
          int o[3] = {0, 0, 0};
          for (int r = 0; r < D; ++r) o[r] = node_off(D, sg, j, r, P) - node_off(D, sg, i, r, P);
          int pos = 0;
          bool found = false;
          for (; pos < n[k]; ++pos) {
            const int c = compare(off[k][pos], o);
            if (c == 0) found = true;
            if (c >= 0) break;
          }
          if (found) continue;
          for (int t = n[k]; t > pos; --t)
            for (int r = 0; r < 3; ++r) off[k][t][r] = off[k][t - 1][r];
          for (int r = 0; r < 3; ++r) off[k][pos][r] = o[r];
          ++n[k];
        }
      }
    for (int k = 0; k < NCLS; ++k) {
      start[k + 1] = start[k] + n[k];
      const int z[3] = {0, 0, 0};
      for (int e = 0; e < n[k]; ++e)
        if (compare(off[k][e], z) == 0) centre[k] = e;
    }
  }
  // class of local node i of the simplex sg in a cell at the lattice origin
  __host__ __device__ static constexpr int class_of_node(int sg, int i) {
    int k = 0;
    for (int r = 0; r < D; ++r) k |= (node_off(D, sg, i, r, P) % P) << r;
    return k;
  }
  __host__ __device__ static constexpr int compare(const int* a, const int* b) {
    for (int r = 0; r < 3; ++r)
      if (a[r] != b[r]) return a[r] < b[r] ? -1 : 1;
    return 0;
  }
  __host__ __device__ constexpr int total() const { return start[NCLS]; }
};
// One shape per (D, P).  Device code reads it only through the integral
// constants below (template arguments), so it sees plain constants.
template <int D, int P>
struct Shape {
  static constexpr StencilShape<D, P> s{};
};
template <int D, int P, int K, int E, int C>
__host__ __device__ constexpr int shape_off() {
  return std::integral_constant<int, Shape<D, P>::s.off[K][E][C]>::value;
}
template <int D, int P, int K>
__host__ __device__ constexpr int shape_n() {
  return std::integral_constant<int, Shape<D, P>::s.n[K]>::value;
}
template <int D, int P, int K>
__host__ __device__ constexpr int shape_start() {
  return std::integral_constant<int, Shape<D, P>::s.start[K]>::value;
}
template <int D, int P, int K>
__host__ __device__ constexpr int shape_centre() {
  return std::integral_constant<int, Shape<D, P>::s.centre[K]>::value;
}
template <int D, int P>
__host__ __device__ constexpr int shape_total() {
  return std::integral_constant<int, Shape<D, P>::s.start[StencilShape<D, P>::NCLS]>::value;
}

template <class R>
__device__ __forceinline__ R fma_r(R a, R b, R c);
template <>
__device__ __forceinline__ float fma_r<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_r<double>(double a, double b, double c) { return fma(a, b, c); }

// Row sum of class K at storage slot `slot`: sum over the class's offsets, in
// their fixed order, of weight * x at the neighbour.  d0 / d1: packed-index
// increments of the two slower axes for offsets -P..P (the fastest axis adds
// its offset itself).
template <int D, class R, int P, int K, int... E>
__device__ __forceinline__ R stencil_row(std::integer_sequence<int, E...>, const R* W, const R* __restrict__ x,
                                         int64_t slot, const int* d0, const int* d1) {
  constexpr int S0 = shape_start<D, P, K>();
  R v = R(0);
  if constexpr (D == 3)
    ((v = fma_r<R>(W[S0 + E],
                   __ldg(x + slot + (d0[shape_off<D, P, K, E, 0>() + P] + d1[shape_off<D, P, K, E, 1>() + P] +
                                     shape_off<D, P, K, E, 2>())),
                   v)),
     ...);
  else
    ((v = fma_r<R>(W[S0 + E], __ldg(x + slot + (d0[shape_off<D, P, K, E, 0>() + P] + shape_off<D, P, K, E, 1>())), v)),
     ...);
  return v;
}
template <int D, class R, int P, int MODE, int K = 0>
__device__ __forceinline__ R stencil_node(int k, const R* W, const R* __restrict__ x, int64_t slot, const int* d0,
                                          const int* d1) {
  if constexpr (K + 1 < StencilShape<D, P>::NCLS) {
    if (k != K) return stencil_node<D, R, P, MODE, K + 1>(k, W, x, slot, d0, d1);
  }
  if constexpr (MODE == kOpDiag) {
    constexpr int c = shape_start<D, P, K>() + shape_centre<D, P, K>();
    return W[c];
  } else {
    return stencil_row<D, R, P, K>(std::make_integer_sequence<int, shape_n<D, P, K>()>{}, W, x, slot, d0, d1);
  }
}

// Sum over the block (fixed shuffle tree, so deterministic); valid in thread
// 0.  sh holds one value per warp; callers separate two sums by a barrier.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = int(threadIdx.x) < int(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Completes a CG reduction inside the kernel that produced its last
// partials: every block has written its partial(s) (thread 0, before this
// call); the last block to arrive sums part[0 .. nparts) (what = 2: and
// part[nparts .. 2 nparts)) in a fixed order, so the result does not depend
// on which block is last, updates the scalars and resets the arrival count.
// No block waits for another.
__device__ void finish_cg(const double* part, int nparts, int what, Scalars* sc, double* sh) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&sc->arrived, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // eight independent loads in flight per thread; the grouping is fixed
  double s1 = 0.0, s2 = 0.0;
  const int step = int(blockDim.x);
  for (int i0 = threadIdx.x; i0 < nparts; i0 += 8 * step) {
    double v1[8], v2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * step;
      v1[j] = i < nparts ? __ldcg(part + i) : 0.0;
      v2[j] = (what == 2 && i < nparts) ? __ldcg(part + nparts + i) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      s1 += v1[j];
      s2 += v2[j];
    }
  }
  const double a = block_sum(s1, sh);
  __syncthreads();
  const double b = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    cg_scalars_update(what, a, b, sc);
    sc->arrived = 0;
  }
}

struct StencilArgs {
  const void* wtab;       // per macro: mass weights, then stiffness weights ([2][entries])
  const uint32_t* nodes;  // interior lattice points, packed (3D: q0 | q1 << 10 | q2 << 20; 2D: q0 | q1 << 16)
  const int4* items;      // (macro, class, first node, count); 4 per group, one macro per group
  int64_t n_groups;
  int npm;
  Scalars* sc;
  int finish;             // kOpCg: > 0 when this pass completes the p.q reduction over `finish` partials
};

// The stencil pass over the interior nodes: each warp takes up to 32 nodes
// of one class of one macro (consecutive in the class's list, which follows
// the storage order), each lane one node; a block takes groups of 4 such
// items of one macro (persistent over the groups), with that macro's weights
// scale (Wm + alpha Wa) in shared memory.  kOpCg leaves one partial of p.q
// per block in part[blockIdx.x].
template <int D, class R, int P, int MODE>
__global__ void __launch_bounds__(128) k_stencil(StencilArgs a, const R* __restrict__ x, R* __restrict__ y, R alpha,
                                                 R scale, double* part) {
  constexpr int NT = shape_total<D, P>();
  __shared__ R W[NT];
  __shared__ double sh[4];
  if (a.sc != nullptr && a.sc->done) return;  // uniform over the grid
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  R pq = R(0);
  int cur = -1;
  for (int64_t g = blockIdx.x; g < a.n_groups; g += gridDim.x) {
    const int m = a.items[g * 4].x;  // the group's macro (uniform over the block)
    if (m != cur) {
      __syncthreads();
      const R* tab = static_cast<const R*>(a.wtab) + size_t(m) * 2 * NT;
      for (int t = threadIdx.x; t < NT; t += blockDim.x) W[t] = scale * (tab[t] + alpha * tab[NT + t]);
      __syncthreads();
      cur = m;
    }
    const int4 it = a.items[g * 4 + warp];
    if (lane >= it.w) continue;
    const uint32_t pk = a.nodes[it.z + lane];
    const int q0 = D == 3 ? int(pk & 1023u) : int(pk & 0xFFFFu);
    const int q1 = D == 3 ? int((pk >> 10) & 1023u) : int(pk >> 16);
    const int q2 = D == 3 ? int(pk >> 20) : 0;
    const int64_t slot = int64_t(m) * a.npm + (D == 3 ? tri3d(q0) + tri2d(q1) + q2 : tri2d(q0) + q1);
    int d0[2 * P + 1], d1[2 * P + 1];
#pragma unroll
    for (int o = -P; o <= P; ++o) {
      d0[o + P] = D == 3 ? tri3d(q0 + o) - tri3d(q0) : tri2d(q0 + o) - tri2d(q0);
      d1[o + P] = D == 3 ? tri2d(q1 + o) - tri2d(q1) : 0;
    }
    const R v = stencil_node<D, R, P, MODE>(it.y, W, x, slot, d0, d1);
    if constexpr (MODE == kOpCg) {
      y[slot] = v;
      pq = fma_r<R>(x[slot], v, pq);  // interior nodes: owners, never on the boundary
    } else {
      y[slot] += v;
    }
  }
  if constexpr (MODE == kOpCg) {
    __syncthreads();
    const double t = block_sum(double(pq), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (a.finish > 0) finish_cg(part, a.finish, 1, a.sc, sh);
  }
}

struct FaceRows {
  const int* off;        // row r: entries [off[r], off[r + 1])
  const int* col;        // column: a storage slot of the neighbour
  const void* w;         // [2][nnz]: mass weights, then stiffness weights
  int64_t nnz;
  const int* copy_off;   // row r's node: storage copies [copy_off[r], copy_off[r + 1]), owner first
  const int* copies;
  int64_t n;             // rows
  Scalars* sc;
  int finish;            // kOpCg: > 0 when this pass completes the p.q reduction over `finish` partials
  double* part0;         // start of the reduction space (the stencil's partials come first)
};

// The assembled rows of the face nodes off the Dirichlet boundary (nodes on a
// face shared by two or more macros): one warp per row, lane e taking
// entries e, e + 32, ..., then a butterfly sum (every lane ends with the same
// bits, so any lane may write).  The row's value goes to every storage copy
// of its node.  kOpCg: y = v and a partial of p.q per block (p = x at the
// owner copy); kOpDiag: the entry whose column is the owner copy.
template <class R, int MODE>
__global__ void __launch_bounds__(kRedThreads) k_face_rows(FaceRows a, const R* __restrict__ x, R* __restrict__ y,
                                                           R alpha, R scale, double* part) {
  __shared__ double sh[kRedThreads / 32];
  if (a.sc != nullptr && a.sc->done) return;
  const int lane = int(threadIdx.x) & 31;
  const int64_t w0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const R* wm = static_cast<const R*>(a.w);
  const R* wa = wm + a.nnz;
  R pq = R(0);
  for (int64_t r = w0; r < a.n; r += nw) {
    const int e0 = a.off[r], e1 = a.off[r + 1];
    const int c0 = a.copy_off[r], c1 = a.copy_off[r + 1];
    const int self = a.copies[c0];
    R v = R(0);
    for (int e = e0 + lane; e < e1; e += 32) {
      const R wt = scale * fma_r<R>(alpha, __ldg(wa + e), __ldg(wm + e));
      const int c = __ldg(a.col + e);
      if constexpr (MODE == kOpDiag) {
        if (c == self) v += wt;
      } else {
        v = fma_r<R>(wt, __ldg(x + c), v);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    for (int k = c0 + lane; k < c1; k += 32) {
      if constexpr (MODE == kOpCg) y[a.copies[k]] = v;
      else y[a.copies[k]] += v;
    }
    if (MODE == kOpCg && lane == 0) pq = fma_r<R>(x[self], v, pq);
  }
  if constexpr (MODE == kOpCg) {
    const double t = block_sum(double(pq), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (a.finish > 0) finish_cg(a.part0, a.finish, 1, a.sc, sh);
  }
}

// ys[colour][slot] = scale (M + alpha A) x summed over the simplices of one
// cell that lie in the macro, for every node of the cell's (P + 1)^d node
// box, into the accumulators of the cell's colour (no two cells of one colour
// share a node, so a store suffices).
// The cell's x values are gathered once and its sums kept in registers (the
// simplex loop is unrolled, so every local node index is a constant).  DIAG:
// only the diagonal (x unused).  BL: the mesh is blended (2D) and every micro
// simplex has its own tables (blended_element_tables) instead of one per
// orientation and macro.
template <int D, class R, int P, bool DIAG, bool BL = false>
__global__ void __launch_bounds__(kDiffThreads) k_apply(OpArgs a, const R* __restrict__ x, R* __restrict__ ys_all,
                                                        R alpha, R scale) {
  constexpr int NB = n_local(D, P);
  constexpr int NP = n_perm(D);
  constexpr int TAB = NB * NB * (1 + NP);
  constexpr int W = P + 1;
  constexpr int NC = D == 3 ? W * W * W : W * W;
  __shared__ R E[BL ? 1 : NP][NB * NB];  // M + alpha A_sigma of the block's macro
  if (a.sc != nullptr && a.sc->done) return;  // uniform over the grid
  const int4 ck = a.chunks[blockIdx.x];
  constexpr int NCOL = 1 << D;
  R* ys = ys_all + 32 * ck.w;  // + (slot / 32) 32 NCOL + slot % 32
  if constexpr (!BL) {
    const R* tab = static_cast<const R*>(a.tables) + size_t(ck.x) * TAB;
    for (int t = threadIdx.x; t < NP * NB * NB; t += blockDim.x) {
      const int sg = t / (NB * NB), e = t - sg * NB * NB;
      E[sg][e] = scale * (tab[e] + alpha * tab[NB * NB * (1 + sg) + e]);
    }
    __syncthreads();
  }
  if (int(threadIdx.x) >= ck.z) return;
  const int4 cv = a.cellv[ck.y + int(threadIdx.x)];
  const int c[3] = {cv.x, cv.y, cv.z};
  const int64_t base = int64_t(ck.x) * a.npm;
  // the cell's node box: slots (nodes outside the macro's reference simplex,
  // p1 >= p2 [>= p3], do not exist and stay untouched)
  int64_t sl[NC];
  bool ex[NC];
  R xc[NC], acc[NC];
#pragma unroll
  for (int l = 0; l < NC; ++l) {
    const int i0 = D == 3 ? l / (W * W) : l / W;
    const int i1 = D == 3 ? (l / W) % W : l % W;
    const int i2 = D == 3 ? l % W : 0;
    const int q0 = P * c[0] + i0, q1 = P * c[1] + i1, q2 = D == 3 ? P * c[2] + i2 : 0;
    ex[l] = q0 >= q1 && (D == 2 || q1 >= q2);
    sl[l] = base + (D == 3 ? tri3d(q0) + tri2d(q1) + q2 : tri2d(q0) + q1);
    xc[l] = (!DIAG && ex[l]) ? x[sl[l]] : R(0);
    acc[l] = R(0);
  }
#pragma unroll
  for (int sg = 0; sg < NP; ++sg) {
    // the simplex lies in the macro's reference simplex iff axes with equal
    // cell coordinates keep their order (a before b for a < b)
    bool inside = true;
#pragma unroll
    for (int u = 0; u < D; ++u)
#pragma unroll
      for (int v = u + 1; v < D; ++v)
        if (c[perm_axis(D, sg, u)] == c[perm_axis(D, sg, v)] && perm_axis(D, sg, u) > perm_axis(D, sg, v))
          inside = false;
    if (!inside) continue;
    const R* te = nullptr;
    if constexpr (BL) {
      // the simplex's own tables: [M | A] after the cells before it
      const int64_t ncell = int64_t(a.N) * (a.N + 1) / 2;
      te = static_cast<const R*>(a.tables) + ((int64_t(ck.x) * ncell + tri2d(c[0]) + c[1]) * NP + sg) * 2 * NB * NB;
    }
#pragma unroll
    for (int ii = 0; ii < NB; ++ii) {
      R v = R(0);
      if (DIAG) {
        v = BL ? scale * (te[ii * NB + ii] + alpha * te[NB * NB + ii * NB + ii]) : E[sg][ii * NB + ii];
      } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const R e = BL ? scale * (te[ii * NB + j] + alpha * te[NB * NB + ii * NB + j]) : E[sg][ii * NB + j];
          v += e * xc[local_index<D, P>(sg, j)];
        }
      }
      acc[local_index<D, P>(sg, ii)] += v;
    }
  }
#pragma unroll
  for (int l = 0; l < NC; ++l)
    if (ex[l]) ys[(sl[l] >> 5) * (32 * NCOL) + (sl[l] & 31)] = acc[l];
}

// The fold of the cell pass: for every fold node f, the sum over its
// storage copies (ascending slot order: off / slots) of their NCOL colour
// accumulators (ascending colour), applied to every copy (kOpAccum / kOpDiag:
// y += v; kOpCg: y = v, 0 on the boundary, with a partial of p.q per block
// in part[blockIdx.x], p = x at the node's first copy).
template <class R, int NCOL, int MODE>
__global__ void __launch_bounds__(kRedThreads) k_fold_nodes(const R* __restrict__ ys, R* __restrict__ y,
                                                            const int* __restrict__ off, const int* __restrict__ slots,
                                                            const uint8_t* __restrict__ fbnd, int64_t nf,
                                                            const R* __restrict__ x, double* part, Scalars* sc) {
  __shared__ double sh[kRedThreads / 32];
  if (sc != nullptr && sc->done) return;
  R pq = R(0);
  for (int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < nf; f += int64_t(gridDim.x) * blockDim.x) {
    const int k0 = off[f], k1 = off[f + 1];
    R v = R(0);
    for (int k = k0; k < k1; ++k) {
      const int sl = slots[k];
      const R* e = ys + int64_t(sl >> 5) * (32 * NCOL) + (sl & 31);
      R w[NCOL];
#pragma unroll
      for (int c = 0; c < NCOL; ++c) w[c] = __ldg(e + 32 * c);
#pragma unroll
      for (int c = 0; c < NCOL; ++c) v += w[c];
    }
    if constexpr (MODE == kOpCg) {
      if (fbnd[f]) v = R(0);
      for (int k = k0; k < k1; ++k) y[slots[k]] = v;
      pq = fma_r<R>(x[slots[k0]], v, pq);
    } else {
      for (int k = k0; k < k1; ++k) y[slots[k]] += v;
    }
  }
  if constexpr (MODE == kOpCg) {
    const double t = block_sum(double(pq), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    finish_cg(part, int(gridDim.x), 1, sc, sh);
  }
}

// ---------------------------------------------------------------------------
// Device: CG vector kernels and deterministic reductions (per-block partials
// in a fixed order, then one block sums the partials in a fixed order).  The
// vectors are in the storage layout: the copies of an interface node hold the
// same value, and the dot products count each interior unknown once (act: the
// owner copy of a node off the Dirichlet boundary).
// ---------------------------------------------------------------------------

// r := r with zero boundary; z = dinv r; p = z; q = 0; partials (r.z, r.r).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_start(R* r, R* z, R* p, R* q, const R* dinv, const uint8_t* bnd,
                                                          const uint8_t* act, int64_t n, double* part) {
  __shared__ double sh[kRedThreads / 32];
  // per-thread partials in the working precision (a few terms each), summed in FP64
  R rz = R(0), rr = R(0);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    R ri = bnd[i] ? R(0) : r[i];
    r[i] = ri;
    const R zi = dinv[i] * ri;
    z[i] = zi;
    p[i] = zi;
    q[i] = R(0);
    if (act[i]) {
      rz += ri * zi;
      rr += ri * ri;
    }
  }
  const double s1 = block_sum(double(rz), sh);
  __syncthreads();
  const double s2 = block_sum(double(rr), sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

// x += alpha p; r -= alpha q; z = dinv r; partials (r.z, r.r), and the last
// block completes the reduction (beta, the iteration count, the done flag).
// Each thread takes kVec elements a grid stride apart per round (their loads
// independent, so they are in flight together).
constexpr int kVec = 4;

template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(R* x, R* r, R* z, const R* p, const R* q, const R* dinv,
                                                           const uint8_t* act, Scalars* sc, int64_t n, double* part) {
  __shared__ double sh[kRedThreads / 32];
  if (sc->done) return;
  const R al = R(sc->alpha);
  R rz = R(0), rr = R(0);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
    R pv[kVec], qv[kVec], rv[kVec], dv[kVec], xv[kVec];
    bool av[kVec];
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
      const int64_t i = i0 + j * stride;
      const bool in = i < n;
      pv[j] = in ? p[i] : R(0);
      qv[j] = in ? q[i] : R(0);
      rv[j] = in ? r[i] : R(0);
      dv[j] = in ? dinv[i] : R(0);
      xv[j] = in ? x[i] : R(0);
      av[j] = in && act[i];
    }
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
      const int64_t i = i0 + j * stride;
      if (i >= n) continue;
      x[i] = xv[j] + al * pv[j];
      const R ri = rv[j] - al * qv[j];
      r[i] = ri;
      const R zi = dv[j] * ri;
      z[i] = zi;
      if (av[j]) {
        rz += ri * zi;
        rr += ri * ri;
      }
    }
  }
  const double s1 = block_sum(double(rz), sh);
  __syncthreads();
  const double s2 = block_sum(double(rr), sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
  finish_cg(part, int(gridDim.x), 2, sc, sh);
}

// p = z + beta p (q is overwritten by the next operator pass).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_direction(R* p, const R* z, const Scalars* sc, int64_t n) {
  if (sc->done) return;
  const R be = R(sc->beta);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
    R zv[kVec], pv[kVec];
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
      const int64_t i = i0 + j * stride;
      zv[j] = i < n ? z[i] : R(0);
      pv[j] = i < n ? p[i] : R(0);
    }
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
      const int64_t i = i0 + j * stride;
      if (i < n) p[i] = zv[j] + be * pv[j];
    }
  }
}

// Starts a CG run: sums the partials of k_cg_start (r.z, r.r) and sets the
// stopping residual, the iteration budget and the done flag.
__global__ void __launch_bounds__(kRedThreads) k_cg_begin(const double* part, int nparts, Scalars* sc, double stop_rr,
                                                          int budget) {
  __shared__ double sh[kRedThreads / 32];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    s1 += part[i];
    s2 += part[nparts + i];
  }
  const double a = block_sum(s1, sh);
  __syncthreads();
  const double b = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    sc->rz = a;
    sc->rr = b;
    sc->stop_rr = stop_rr;
    sc->budget = budget;
    sc->iters = 0;
    sc->arrived = 0;
    sc->done = (b <= stop_rr || !isfinite(b) || budget <= 0) ? 1 : 0;
  }
}

// |b|^2 over the interior unknowns (the residual reference).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const R* b, const uint8_t* act, int64_t n, double* part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (act[i]) s += double(b[i]) * double(b[i]);
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_into(const double* part, int nparts, double* out) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) *out = t;
}

// dinv = 1 / diag (interior), 0 on the boundary.
template <class R>
__global__ void k_invert_diag(R* d, const uint8_t* bnd, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (bnd[i] || d[i] == R(0)) ? R(0) : R(1) / d[i];
}

// x = where(bnd, v, x)
template <class R>
__global__ void k_set_boundary(R* x, const R* v, const uint8_t* bnd, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && bnd[i]) x[i] = v[i];
}

// r32 = float(r) on the interior, 0 on the boundary; d32 = 0.
__global__ void k_residual_to_float(const double* r, float* r32, float* d32, const uint8_t* bnd, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    r32[i] = bnd[i] ? 0.0f : float(r[i]);
    d32[i] = 0.0f;
  }
}

// x += double(d32) (the correction of one inner solve)
__global__ void k_add_correction(double* x, const float* d32, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) x[i] += double(d32[i]);
}

template <class R>
__global__ void k_copy(R* dst, const R* src, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host: set-up at mesh creation and the solve.
// ---------------------------------------------------------------------------

namespace {

// Node-centred stencil weights of one affine macro from its element tables
// (mass Mt [nb*nb], stiffness At [n_perm][nb*nb]): out[0 .. NT) mass,
// out[NT .. 2 NT) stiffness, in StencilShape order.  Every simplex holding a
// node of class k as its local node i adds its row i at the offsets of the
// other local nodes.
template <int D, int P>
void stencil_weights(const double* Mt, const double* At, double* out) {
  constexpr StencilShape<D, P> S{};
  constexpr int NB = n_local(D, P), NT = S.total();
  std::fill(out, out + 2 * NT, 0.0);
  for (int sg = 0; sg < n_perm(D); ++sg)
    for (int i = 0; i < NB; ++i) {
      const int k = StencilShape<D, P>::class_of_node(sg, i);
      for (int j = 0; j < NB; ++j) {
        int o[3] = {0, 0, 0};
        for (int r = 0; r < D; ++r) o[r] = node_off(D, sg, j, r, P) - node_off(D, sg, i, r, P);
        int e = 0;
        while (e < S.n[k] && StencilShape<D, P>::compare(S.off[k][e], o) != 0) ++e;
        out[S.start[k] + e] += Mt[i * NB + j];
        out[NT + S.start[k] + e] += At[(size_t(sg) * NB + i) * NB + j];
      }
    }
}

int stencil_entries(int d, int p) {
  if (d == 3) return p == 2 ? shape_total<3, 2>() : shape_total<3, 1>();
  return p == 2 ? shape_total<2, 2>() : shape_total<2, 1>();
}

// Replaces *dst by a device copy of `bytes` bytes at `data` (nullptr when empty).
bool upload_bytes(void** dst, const void* data, size_t bytes) {
  cudaFree(*dst);
  *dst = nullptr;
  if (bytes == 0) return true;
  return cudaMalloc(dst, bytes) == cudaSuccess && cudaMemcpy(*dst, data, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}
template <class T>
bool upload(T** dst, const std::vector<T>& v) {
  void* p = *dst;
  const bool ok = upload_bytes(&p, v.data(), sizeof(T) * v.size());
  *dst = static_cast<T*>(p);
  return ok;
}
// A table given in FP64 into an untyped device buffer, in FP64 or rounded to FP32.
bool upload_real(void** dst, const std::vector<double>& v, bool fp64) {
  if (fp64) return upload_bytes(dst, v.data(), sizeof(double) * v.size());
  const std::vector<float> f(v.begin(), v.end());
  return upload_bytes(dst, f.data(), sizeof(float) * f.size());
}

// Lattice point (q0, q1, q2) of every slot of one macro, in storage order.
template <class F>
void for_each_lattice_point(int d, int M, F f) {
  int64_t s = 0;
  if (d == 2) {
    for (int q0 = 0; q0 <= M; ++q0)
      for (int q1 = 0; q1 <= q0; ++q1) f(s++, q0, q1, 0);
  } else {
    for (int q0 = 0; q0 <= M; ++q0)
      for (int q1 = 0; q1 <= q0; ++q1)
        for (int q2 = 0; q2 <= q1; ++q2) f(s++, q0, q1, q2);
  }
}

bool on_macro_face(int d, int M, int q0, int q1, int q2) {
  return d == 3 ? (q0 == M || q0 == q1 || q1 == q2 || q2 == 0) : (q0 == M || q0 == q1 || q1 == 0);
}

// Interior nodes (strictly inside their macro: the stencil pass), as lists
// per macro and class in storage order, and the warp items over them: up to
// 32 nodes of one class each, 4 items of one macro per group (padded with
// empty items).
void interior_lists(const elm_mesh_s* me, std::vector<uint32_t>& nodes, std::vector<int4>& items) {
  const int d = me->dim, P = me->order, M = me->M;
  const int ncls = P == 2 ? (1 << d) : 1;
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const size_t first_item = items.size();
    for (int k = 0; k < ncls; ++k) {
      const size_t first = nodes.size();
      for_each_lattice_point(d, M, [&](int64_t, int q0, int q1, int q2) {
        const bool interior = d == 3 ? (q0 < M && q0 > q1 && q1 > q2 && q2 > 0) : (q0 < M && q0 > q1 && q1 > 0);
        if (!interior) return;
        const int cls = P == 2 ? (d == 3 ? (q0 & 1) | ((q1 & 1) << 1) | ((q2 & 1) << 2) : (q0 & 1) | ((q1 & 1) << 1)) : 0;
        if (cls != k) return;
        nodes.push_back(d == 3 ? uint32_t(q0) | (uint32_t(q1) << 10) | (uint32_t(q2) << 20)
                               : uint32_t(q0) | (uint32_t(q1) << 16));
      });
      for (size_t a = first; a < nodes.size(); a += 32)
        items.push_back(make_int4(int(m), k, int(a), int(std::min<size_t>(32, nodes.size() - a))));
    }
    while ((items.size() - first_item) % 4) items.push_back(make_int4(int(m), 0, 0, 0));
  }
}

// The assembled rows of the face nodes off the Dirichlet boundary (the nodes
// on a face shared with another macro): every micro simplex holding such a
// node as its local node i adds its element row i (mass and stiffness) at the
// owner slots of its other local nodes; equal columns are summed (in the
// order of the cells, then simplices), and the columns sorted by unique id.
struct RowsHost {
  std::vector<int> off{0}, col, copy_off{0}, copies;
  std::vector<double> wm, wa;
};
RowsHost face_rows(const elm_mesh_s* me, const std::vector<double>& t64) {
  const int d = me->dim, P = me->order, N = me->N, M = me->M, nb = n_local(d, P), np = n_perm(d);
  const size_t tab = size_t(nb) * nb * (1 + np);
  std::vector<uint8_t> face_slot(me->n_storage, 0);
  for (int64_t m = 0; m < me->n_macros; ++m)
    for_each_lattice_point(d, M, [&](int64_t s, int q0, int q1, int q2) {
      if (on_macro_face(d, M, q0, q1, q2)) face_slot[m * me->npm + s] = 1;
    });
  std::vector<int64_t> rid(me->n_unique, -1);
  int64_t nrows = 0;
  RowsHost h;
  for (int64_t u = 0; u < me->n_unique; ++u)
    if (face_slot[me->owner[u]] && !me->dbnd[u]) rid[u] = nrows++;
  struct Raw {
    int64_t row, colu;
    double m, a;
  };
  std::vector<Raw> raw;
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const double* Mt = t64.data() + m * tab;
    const double* At = Mt + size_t(nb) * nb;
    const int64_t base = m * me->npm;
    for (int c0 = 0; c0 < N; ++c0)
      for (int c1 = 0; c1 <= c0; ++c1)
        for (int c2 = 0; c2 <= (d == 3 ? c1 : 0); ++c2) {
          const int c[3] = {c0, c1, c2};
          for (int sg = 0; sg < np; ++sg) {
            int s[3] = {0, 1, 2};
            perm_of(d, sg, s);
            bool inside = true;
            for (int a = 0; a < d; ++a)
              for (int b = a + 1; b < d; ++b)
                if (c[s[a]] == c[s[b]] && s[a] > s[b]) inside = false;
            if (!inside) continue;
            int64_t u[10];
            bool any = false;
            for (int j = 0; j < nb; ++j) {
              int q[3] = {0, 0, 0};
              for (int r = 0; r < d; ++r) q[r] = P * c[r] + node_off(d, sg, j, r, P);
              const int64_t sl = base + (d == 3 ? int64_t(q[0]) * (q[0] + 1) * (q[0] + 2) / 6 +
                                                      int64_t(q[1]) * (q[1] + 1) / 2 + q[2]
                                                : int64_t(q[0]) * (q[0] + 1) / 2 + q[1]);
              u[j] = me->unique_map[sl];
              any = any || rid[u[j]] >= 0;
            }
            if (!any) continue;
            for (int i = 0; i < nb; ++i) {
              if (rid[u[i]] < 0) continue;
              for (int j = 0; j < nb; ++j)
                raw.push_back({rid[u[i]], u[j], Mt[i * nb + j], At[(size_t(sg) * nb + i) * nb + j]});
            }
          }
        }
  }
  std::stable_sort(raw.begin(), raw.end(), [](const Raw& x, const Raw& y) {
    return x.row != y.row ? x.row < y.row : x.colu < y.colu;
  });
  int64_t r = 0;
  for (size_t k = 0; k < raw.size();) {
    size_t e = k;
    double wm = 0.0, wa = 0.0;
    for (; e < raw.size() && raw[e].row == raw[k].row && raw[e].colu == raw[k].colu; ++e) {
      wm += raw[e].m;
      wa += raw[e].a;
    }
    for (; r < raw[k].row; ++r) h.off.push_back(int(h.col.size()));
    h.col.push_back(int(me->owner[raw[k].colu]));
    h.wm.push_back(wm);
    h.wa.push_back(wa);
    k = e;
  }
  for (; r < nrows; ++r) h.off.push_back(int(h.col.size()));
  // copies of each row's node, owner first (ascending slot; the owner is the lowest)
  std::vector<int64_t> row_of_slot(me->n_storage, -1);
  std::vector<int> cnt(nrows + 1, 0);
  for (int64_t sl = 0; sl < me->n_storage; ++sl) {
    const int64_t rr = rid[me->unique_map[sl]];
    if (rr >= 0) ++cnt[rr + 1];
  }
  for (int64_t k = 0; k < nrows; ++k) cnt[k + 1] += cnt[k];
  h.copy_off.assign(cnt.begin(), cnt.end());
  h.copies.assign(cnt.back(), 0);
  for (int64_t sl = 0; sl < me->n_storage; ++sl) {
    const int64_t rr = rid[me->unique_map[sl]];
    if (rr >= 0) h.copies[cnt[rr]++] = int(sl);
  }
  return h;
}

// Blended meshes: the cell pass over every cell (chunks of at most
// kDiffThreads cells of one colour and one macro, by colour, then macro) and
// its fold into every node.
bool build_cells_and_fold(elm_mesh_s* me) {
  const int d = me->dim, N = me->N;
  const int ncol = 1 << d;
  std::vector<int4> cells, cellv;
  for (int col = 0; col < ncol; ++col)
    for (int64_t m = 0; m < me->n_macros; ++m) {
      const int64_t first = int64_t(cellv.size());
      for (int c0 = col & 1; c0 < N; c0 += 2)
        for (int c1 = (col >> 1) & 1; c1 <= c0; c1 += 2) {
          if (d == 2) {
            cellv.push_back(make_int4(c0, c1, 0, 0));
            continue;
          }
          for (int c2 = (col >> 2) & 1; c2 <= c1; c2 += 2) cellv.push_back(make_int4(c0, c1, c2, 0));
        }
      const int64_t last = int64_t(cellv.size());
      for (int64_t c = first; c < last; c += kDiffThreads)
        cells.push_back(make_int4(int(m), int(c), int(std::min<int64_t>(kDiffThreads, last - c)), col));
    }
  me->n_cell_chunks = int64_t(cells.size());
  std::vector<int> foff(me->n_unique + 1, 0), fslots(me->n_storage);
  for (int64_t sl = 0; sl < me->n_storage; ++sl) ++foff[me->unique_map[sl] + 1];
  for (int64_t u = 0; u < me->n_unique; ++u) foff[u + 1] += foff[u];
  {
    std::vector<int> next(foff.begin(), foff.end() - 1);
    for (int64_t sl = 0; sl < me->n_storage; ++sl) fslots[next[me->unique_map[sl]]++] = int(sl);
  }
  me->n_dface = me->n_unique;
  // the colour accumulators, tiled by 32 slots; zero where no cell of the
  // colour ever writes
  const size_t ysn = size_t((me->n_storage + 31) / 32 * 32) * size_t(ncol);
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  cudaFree(me->d_dys);
  me->d_dys = nullptr;
  return upload(&me->d_dcells, cells) && upload(&me->d_dcellv, cellv) && upload(&me->d_dfold_off, foff) &&
         upload(&me->d_dfold_slots, fslots) && upload(&me->d_dfbnd, me->dbnd) &&
         cudaMalloc(&me->d_dys, ysn * es) == cudaSuccess && cudaMemset(me->d_dys, 0, ysn * es) == cudaSuccess;
}

}  // namespace

namespace {

// Everything the affine operator needs, built on the host: element tables
// and stencil weights per macro, the Dirichlet mask, per-slot masks, the
// interior lists and the face rows.
struct DiffusionHost {
  std::vector<double> t64, w64;
  std::vector<uint8_t> dbnd, bnd_s, act;
  std::vector<int64_t> slot_owner;
  std::vector<uint32_t> nodes;
  std::vector<int4> items;
  RowsHost rows;
};

DiffusionHost diffusion_host(elm_mesh_s* me) {
  DiffusionHost h;
  // the interior lists pack lattice coordinates into 10 bits (3D) or 16 bits
  // (2D) each; the level limits of elm_mesh_create keep M within both
  const int d = me->dim, p = me->order, nb = n_local(d, p), np = n_perm(d);
  const size_t tab = size_t(nb) * nb * (1 + np);
  h.t64.assign(tab * me->n_macros, 0.0);
  for (int64_t m = 0; m < me->n_macros; ++m)
    element_tables(d, p, me->N, me->geo[m], h.t64.data() + m * tab, h.t64.data() + m * tab + size_t(nb) * nb);
  const int nt = stencil_entries(d, p);
  h.w64.assign(size_t(2) * nt * me->n_macros, 0.0);
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const double* Mt = h.t64.data() + m * tab;
    const double* At = Mt + size_t(nb) * nb;
    double* w = h.w64.data() + size_t(2) * nt * m;
    if (d == 3) {
      if (p == 2) stencil_weights<3, 2>(Mt, At, w);
      else stencil_weights<3, 1>(Mt, At, w);
    } else {
      if (p == 2) stencil_weights<2, 2>(Mt, At, w);
      else stencil_weights<2, 1>(Mt, At, w);
    }
  }
  // boundary unknowns: a node on face k (barycentric weight k = 0) of a macro
  // whose face k has no neighbour
  h.dbnd.assign(me->n_unique, 0);
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const MacroGeo& g = me->geo[m];
    for_each_lattice_point(d, me->M, [&](int64_t s, int q0, int q1, int q2) {
      const int pp[5] = {me->M, q0, q1, d == 3 ? q2 : 0, 0};
      bool on = false;
      for (int k = 0; k <= d; ++k) {
        const int w = (d == 3 || k < d) ? pp[k] - pp[k + 1] : pp[k];
        if (w == 0 && g.nb[k] < 0) on = true;
      }
      if (on) h.dbnd[me->unique_map[m * me->npm + s]] = 1;
    });
  }
  me->dbnd = h.dbnd;
  // per slot: boundary, dot-product mask (owner copy, off the boundary), owner slot
  h.bnd_s.assign(me->n_storage, 0);
  h.act.assign(me->n_storage, 0);
  h.slot_owner.assign(me->n_storage, 0);
  for (int64_t sl = 0; sl < me->n_storage; ++sl) {
    const int64_t u = me->unique_map[sl];
    h.bnd_s[sl] = h.dbnd[u];
    h.act[sl] = (me->owner[u] == sl && !h.dbnd[u]) ? 1 : 0;
    h.slot_owner[sl] = me->owner[u];
  }
  interior_lists(me, h.nodes, h.items);
  h.rows = face_rows(me, h.t64);
  return h;
}

}  // namespace

elm_status build_diffusion(elm_mesh_s* me, std::string* err) {
  // packed interior lattice points (10 bits per coordinate in 3D, 16 in 2D)
  // and 32-bit slot columns; elm_mesh_create's level limits keep both
  if ((me->dim == 3 && me->M > 1023) || me->M > 65535 || me->n_storage > int64_t(INT32_MAX) / 2) {
    *err = "diffusion: mesh too large for the solver's 32-bit tables";
    return ELM_ERR_ARG;
  }
  const DiffusionHost h = diffusion_host(me);
  me->n_ditems = int64_t(h.items.size());
  me->n_drows = int64_t(h.rows.off.size()) - 1;
  me->n_dnnz = int64_t(h.rows.col.size());
  std::vector<double> rw(h.rows.wm);
  rw.insert(rw.end(), h.rows.wa.begin(), h.rows.wa.end());
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&me->n_dsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    *err = std::string("diffusion set-up: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  auto put = [](void** dst, const std::vector<double>& v, bool fp64) { return upload_real(dst, v, fp64); };
  const bool f64 = me->precision == ELM_FP64;
  bool ok = put(&me->d_dtab, h.t64, f64) && put(&me->d_dwtab, h.w64, f64) && put(&me->d_drow_w, rw, f64);
  if (f64)  // FP32 copies for the inner solves of the mixed-precision form
    ok = ok && put(&me->d_dtab32, h.t64, false) && put(&me->d_dwtab32, h.w64, false) &&
         put(&me->d_drow_w32, rw, false);
  ok = ok && upload(&me->d_dnodes, h.nodes) && upload(&me->d_ditems, h.items) && upload(&me->d_drow_off, h.rows.off) &&
       upload(&me->d_drow_col, h.rows.col) && upload(&me->d_drow_copy_off, h.rows.copy_off) &&
       upload(&me->d_drow_copies, h.rows.copies);
  ok = ok && upload(&me->d_dbnd_s, h.bnd_s) && upload(&me->d_dact, h.act) && upload(&me->d_dslot_owner, h.slot_owner);
  ok = ok && cudaMalloc(&me->d_dvec, size_t(kDiffVectors) * me->n_storage * es) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dpart, sizeof(double) * 2 * kRedMaxBlocks) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dscal, sizeof(Scalars) + 2 * sizeof(double)) == cudaSuccess;
  if (f64) ok = ok && cudaMalloc(&me->d_dvec32, size_t(kDiffVectors32) * me->n_storage * 4) == cudaSuccess;
  if (!ok) {
    *err = std::string("diffusion tables: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  me->n_boundary = 0;
  for (uint8_t b : me->dbnd) me->n_boundary += b;
  return ELM_OK;
}

elm_status build_diffusion_blended(elm_mesh_s* me, std::string* err) {
  std::vector<double> t;
  blended_element_tables(me, t);
  if (!upload_real(&me->d_dtab_el, t, true) || !build_cells_and_fold(me)) {
    *err = std::string("blended diffusion tables: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  return ELM_OK;
}

namespace {

// Grids of the operator passes: persistent blocks, at most 8 per SM for the
// face rows and 12 for the stencil pass (its registers allow 12 resident
// 128-thread blocks; measured 4.54 against 4.64 ms for the level-6 FP64 solve
// with 8), so the partials of one reduction stay a few thousand.
inline int capped_blocks(const elm_mesh_s* me, int64_t want) {
  const int64_t cap = 8 * int64_t(me->n_dsm > 0 ? me->n_dsm : 1);
  return int(want < cap ? want : cap);
}
// the stencil pass (affine meshes), then the face rows or, on a blended
// mesh, the cell pass's fold: blocks of each, in launch order
inline int stencil_blocks(const elm_mesh_s* me) {
  if (me->blend.nsec > 0 || me->n_ditems == 0) return 0;
  const int64_t groups = me->n_ditems / 4, cap = 12 * int64_t(me->n_dsm > 0 ? me->n_dsm : 1);
  return int(groups < cap ? groups : cap);
}
inline int second_blocks(const elm_mesh_s* me) {
  if (me->blend.nsec > 0) return me->n_dface > 0 ? red_blocks(me->n_dface) : 0;
  return me->n_drows > 0 ? capped_blocks(me, (me->n_drows + kRedThreads / 32 - 1) / (kRedThreads / 32)) : 0;
}

// The passes of one application, in order.  Affine meshes: the stencil over
// the interior nodes, then the assembled face rows; blended meshes: the cell
// pass into the colour accumulators, then their fold.  MODE (OpMode) says
// what is done with the result; with kOpCg the partials of p.q are left in
// part[0 .. stencil_blocks + second_blocks), and the last pass completes the
// reduction (alpha).  The FP32 inner solves of an FP64 mesh use the FP32
// copies of the weights.
template <class R, int MODE>
cudaError_t launch_op(const elm_mesh_s* me, const R* x, R* y, double alpha, double scale, cudaStream_t s,
                      Scalars* sc, double* part) {
  const R al = R(alpha), sca = R(scale);
  if (me->blend.nsec > 0) {
    if constexpr (sizeof(R) == 8) {  // 2D FP64 only (elm_mesh_set_annulus)
      OpArgs a{me->d_dtab_el, me->d_dcells, me->d_dcellv, int(me->npm), me->N, sc};
      R* ys = static_cast<R*>(me->d_dys);
      constexpr bool DG = MODE == kOpDiag;
      const unsigned g = unsigned(me->n_cell_chunks);
      if (g > 0) {
        if (me->order == 2) k_apply<2, R, 2, DG, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
        else k_apply<2, R, 1, DG, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
      }
      if (me->n_dface > 0)
        k_fold_nodes<R, 4, MODE><<<second_blocks(me), kRedThreads, 0, s>>>(
            ys, y, me->d_dfold_off, me->d_dfold_slots, me->d_dfbnd, me->n_dface, x, part, sc);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  const bool inner = sizeof(R) == 4 && me->precision == ELM_FP64;  // FP32 inner solves of an FP64 mesh
  const int nsb = stencil_blocks(me), nfb = me->n_drows > 0 ? second_blocks(me) : 0;
  const bool cg = MODE == kOpCg;
  if (nsb > 0) {
    StencilArgs st{inner ? me->d_dwtab32 : me->d_dwtab, me->d_dnodes, me->d_ditems, me->n_ditems / 4, int(me->npm),
                   sc, cg && nfb == 0 ? nsb : 0};
    if (me->dim == 3) {
      if (me->order == 2) k_stencil<3, R, 2, MODE><<<nsb, 128, 0, s>>>(st, x, y, al, sca, part);
      else k_stencil<3, R, 1, MODE><<<nsb, 128, 0, s>>>(st, x, y, al, sca, part);
    } else {
      if (me->order == 2) k_stencil<2, R, 2, MODE><<<nsb, 128, 0, s>>>(st, x, y, al, sca, part);
      else k_stencil<2, R, 1, MODE><<<nsb, 128, 0, s>>>(st, x, y, al, sca, part);
    }
  }
  if (me->n_drows > 0) {
    const FaceRows fr{me->d_drow_off, me->d_drow_col,  inner ? me->d_drow_w32 : me->d_drow_w,
                      me->n_dnnz,      me->d_drow_copy_off, me->d_drow_copies,
                      me->n_drows,     sc,                 cg ? nsb + nfb : 0,
                      part};
    k_face_rows<R, MODE><<<nfb, kRedThreads, 0, s>>>(fr, x, y, al, sca, part ? part + nsb : nullptr);
  }
  return cudaGetLastError();
}

// y += scale (M + alpha A) x (diag: the diagonal only), storage layout.
template <class R>
cudaError_t apply_op(const elm_mesh_s* me, const R* x, R* y, double alpha, double scale, bool diag, cudaStream_t s) {
  return diag ? launch_op<R, kOpDiag>(me, x, y, alpha, scale, s, nullptr, nullptr)
              : launch_op<R, kOpAccum>(me, x, y, alpha, scale, s, nullptr, nullptr);
}

// PCG iterations on the interior from the state of k_cg_start (r, z = D^{-1} r,
// p = z; its partials of r.z and r.r in the reduction space): stops when
// |r|^2 <= stop_rr or after `budget` iterations.  Each iteration is three
// passes: the operator (q = E p; its last kernel completes p.q and alpha),
// the update (x, r, z; its last block completes beta and the done flag) and
// the direction.  The iterations are enqueued in batches of kCheckEvery; once
// the device sets the done flag the kernels after it return at once, so the
// host reads the scalars once per batch.  *done = iterations run, *rr = final
// |r|^2.  Returns false on a CUDA error (message in *err).
constexpr int kCheckEvery = 8;

template <class R>
bool pcg_iterate(const elm_mesh_s* me, R* x, R* r, R* z, R* p, R* qv, const R* dinv, double alpha, double stop_rr,
                 int budget, int* done, double* rr, cudaStream_t s, std::string* err) {
  const int64_t n = me->n_storage;
  double* part = me->d_dpart;
  Scalars* sc = reinterpret_cast<Scalars*>(me->d_dscal);
  const int nred = red_blocks(n);
  const int nupd = red_blocks(n / kVec + 1);
  auto chk = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) *err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  k_cg_begin<<<1, kRedThreads, 0, s>>>(part, nred, sc, stop_rr, budget);
  Scalars h{};
  for (;;) {
    if (!chk(cudaMemcpyAsync(&h, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "read") ||
        !chk(cudaStreamSynchronize(s), "sync"))
      return false;
    if (h.done) break;
    for (int k = 0; k < kCheckEvery; ++k) {
      // q = E p (0 on the boundary), p.q and alpha
      if (!chk(launch_op<R, kOpCg>(me, p, qv, alpha, 1.0, s, sc, part), "apply")) return false;
      k_cg_update<R><<<nupd, kRedThreads, 0, s>>>(x, r, z, p, qv, dinv, me->d_dact, sc, n, part);
      k_cg_direction<R><<<nupd, kRedThreads, 0, s>>>(p, z, sc, n);
    }
  }
  *done = h.iters;
  *rr = h.rr;
  return true;
}

// FP64 meshes (affine macros): defect correction with FP32 inner solves.  The
// residual r = b - E x is formed in FP64; E d = r is solved by the same PCG
// in FP32 (to a relative residual of kInnerRtol) and x += d.  Each correction
// gains about four digits, so a solve to 1e-11 takes three FP64 operator
// applications instead of one per iteration: the FP64 products run on this
// part's narrow FP64 pipe, the FP32 ones on its FP32 pipe.
constexpr double kInnerRtol = 3e-5;

elm_status solve_mixed(elm_mesh_s* me, const void* c_hat, const void* c_bnd, const void* q, void* c_new,
                       double tau, double kappa, double theta, double rtol, int max_iter, int* iters, double* resid,
                       cudaStream_t s, std::string* err) {
  const int64_t n = me->n_storage;
  double* v = static_cast<double*>(me->d_dvec);
  double* x = v;
  double* r = v + n;
  double* tmp = v + 2 * n;
  double* b = v + 5 * n;
  float* w = static_cast<float*>(me->d_dvec32);
  float* r32 = w;
  float* z32 = w + n;
  float* p32 = w + 2 * n;
  float* q32 = w + 3 * n;
  float* d32 = w + 4 * n;
  float* dinv32 = w + 5 * n;
  double* part = me->d_dpart;
  double* bnorm = me->d_dscal + sizeof(Scalars) / sizeof(double);
  double* rnorm = bnorm + 1;
  const size_t bytes = size_t(n) * sizeof(double);
  const unsigned eb = unsigned((n + 255) / 256);
  const int nred = red_blocks(n);
  auto chk = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) *err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  // inputs in the storage layout, every copy taking its owner's value
  if (!chk(launch_gather(ELM_FP64, c_hat, x, me->d_dslot_owner, n, 1, s), "gather c_hat")) return ELM_ERR_CUDA;
  if (!chk(cudaMemsetAsync(b, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<double>(me, x, b, -tau * (1.0 - theta) * kappa, 1.0, false, s), "rhs")) return ELM_ERR_CUDA;
  if (q) {
    if (!chk(launch_gather(ELM_FP64, q, tmp, me->d_dslot_owner, n, 1, s), "gather q")) return ELM_ERR_CUDA;
    if (!chk(apply_op<double>(me, tmp, b, 0.0, tau, false, s), "source")) return ELM_ERR_CUDA;
  }
  if (c_bnd) {
    if (!chk(launch_gather(ELM_FP64, c_bnd, tmp, me->d_dslot_owner, n, 1, s), "gather c_bnd")) return ELM_ERR_CUDA;
    k_set_boundary<double><<<eb, 256, 0, s>>>(x, tmp, me->d_dbnd_s, n);
  }
  const double alpha = tau * theta * kappa;
  if (!chk(cudaMemsetAsync(dinv32, 0, size_t(n) * 4, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<float>(me, nullptr, dinv32, alpha, 1.0, true, s), "diagonal")) return ELM_ERR_CUDA;
  k_invert_diag<float><<<eb, 256, 0, s>>>(dinv32, me->d_dbnd_s, n);
  k_norm2<double><<<nred, kRedThreads, 0, s>>>(b, me->d_dact, n, part);
  k_sum_into<<<1, kRedThreads, 0, s>>>(part, nred, bnorm);
  double hb = 0.0;
  if (!chk(cudaMemcpyAsync(&hb, bnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "read") ||
      !chk(cudaStreamSynchronize(s), "sync"))
    return ELM_ERR_CUDA;
  const double bn = std::sqrt(hb);
  const bool interior = me->n_unique > me->n_boundary;
  int total = 0;
  double rel = 0.0;
  for (int outer = 0;; ++outer) {
    // r = b - E x (FP64), interior only
    k_copy<double><<<eb, 256, 0, s>>>(r, b, n);
    if (!chk(apply_op<double>(me, x, r, alpha, -1.0, false, s), "residual")) return ELM_ERR_CUDA;
    k_norm2<double><<<nred, kRedThreads, 0, s>>>(r, me->d_dact, n, part);
    k_sum_into<<<1, kRedThreads, 0, s>>>(part, nred, rnorm);
    double hr = 0.0;
    if (!chk(cudaMemcpyAsync(&hr, rnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "read") ||
        !chk(cudaStreamSynchronize(s), "sync"))
      return ELM_ERR_CUDA;
    rel = bn > 0.0 ? std::sqrt(hr) / bn : std::sqrt(hr);
    if (!interior || !(rel > rtol) || total >= max_iter || !std::isfinite(rel)) break;
    // inner FP32 solve of E d = r from d = 0
    k_residual_to_float<<<eb, 256, 0, s>>>(r, r32, d32, me->d_dbnd_s, n);
    k_cg_start<float><<<nred, kRedThreads, 0, s>>>(r32, z32, p32, q32, dinv32, me->d_dbnd_s, me->d_dact, n, part);
    int done = 0;
    double rr32 = 0.0;
    // stop at kInnerRtol of the inner start, or where the outer tolerance is met
    const double start_rr = hr;
    const double stop = std::max(kInnerRtol * kInnerRtol * start_rr, 0.25 * rtol * rtol * bn * bn);
    if (!pcg_iterate<float>(me, d32, r32, z32, p32, q32, dinv32, alpha, stop, max_iter - total, &done, &rr32, s, err))
      return ELM_ERR_CUDA;
    total += done;
    k_add_correction<<<eb, 256, 0, s>>>(x, d32, n);
    if (outer > 64) break;  // safeguard: corrections stopped converging
  }
  if (iters) *iters = total;
  if (resid) *resid = rel;
  if (!chk(cudaMemcpyAsync(c_new, x, bytes, cudaMemcpyDeviceToDevice, s), "result")) return ELM_ERR_CUDA;
  if (!std::isfinite(rel)) {
    *err = "non-finite residual";
    return ELM_ERR_NONFINITE;
  }
  if (rel > rtol && interior) {
    *err = "CG did not reach the tolerance within max_iter iterations (relative residual " + std::to_string(rel) + ")";
    return ELM_ERR_NOT_CONVERGED;
  }
  return ELM_OK;
}

template <class R>
elm_status solve(elm_mesh_s* me, const void* c_hat, const void* c_bnd, const void* q, void* c_new, double tau,
                 double kappa, double theta, double rtol, int max_iter, int* iters, double* resid, cudaStream_t s,
                 std::string* err) {
  const int64_t n = me->n_storage;
  R* v = static_cast<R*>(me->d_dvec);
  R* x = v;
  R* r = v + n;
  R* z = v + 2 * n;
  R* p = v + 3 * n;
  R* qv = v + 4 * n;
  R* b = v + 5 * n;
  R* dinv = v + 6 * n;
  double* part = me->d_dpart;
  double* bnorm = me->d_dscal + sizeof(Scalars) / sizeof(double);
  const size_t bytes = size_t(n) * sizeof(R);
  const unsigned eb = unsigned((n + 255) / 256);
  const int nred = red_blocks(n);
  const int prec = me->precision;
  auto chk = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) *err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  // inputs in the storage layout, every copy taking its owner's value; right-hand side b
  if (!chk(launch_gather(prec, c_hat, x, me->d_dslot_owner, n, 1, s), "gather c_hat")) return ELM_ERR_CUDA;
  if (!chk(cudaMemsetAsync(b, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<R>(me, x, b, -tau * (1.0 - theta) * kappa, 1.0, false, s), "rhs")) return ELM_ERR_CUDA;
  if (q) {
    if (!chk(launch_gather(prec, q, z, me->d_dslot_owner, n, 1, s), "gather q")) return ELM_ERR_CUDA;
    if (!chk(apply_op<R>(me, z, b, 0.0, tau, false, s), "source")) return ELM_ERR_CUDA;
  }
  if (c_bnd) {
    if (!chk(launch_gather(prec, c_bnd, z, me->d_dslot_owner, n, 1, s), "gather c_bnd")) return ELM_ERR_CUDA;
    k_set_boundary<R><<<eb, 256, 0, s>>>(x, z, me->d_dbnd_s, n);
  }
  // Jacobi preconditioner of E = M + tau theta kappa A
  const double alpha = tau * theta * kappa;
  if (!chk(cudaMemsetAsync(dinv, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<R>(me, x, dinv, alpha, 1.0, true, s), "diagonal")) return ELM_ERR_CUDA;
  k_invert_diag<R><<<eb, 256, 0, s>>>(dinv, me->d_dbnd_s, n);
  k_norm2<R><<<nred, kRedThreads, 0, s>>>(b, me->d_dact, n, part);
  k_sum_into<<<1, kRedThreads, 0, s>>>(part, nred, bnorm);
  // r = b - E x, restricted to the interior; z = D^{-1} r; p = z
  k_copy<R><<<eb, 256, 0, s>>>(r, b, n);
  if (!chk(apply_op<R>(me, x, r, alpha, -1.0, false, s), "residual")) return ELM_ERR_CUDA;
  k_cg_start<R><<<nred, kRedThreads, 0, s>>>(r, z, p, qv, dinv, me->d_dbnd_s, me->d_dact, n, part);
  double hb = 0.0;
  if (!chk(cudaMemcpyAsync(&hb, bnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "read") ||
      !chk(cudaStreamSynchronize(s), "sync"))
    return ELM_ERR_CUDA;
  const double bn = std::sqrt(hb);
  const bool interior = me->n_unique > me->n_boundary;
  int it = 0;
  double rr = 0.0;
  const double stop = bn > 0.0 ? rtol * rtol * bn * bn : rtol * rtol;
  if (!pcg_iterate<R>(me, x, r, z, p, qv, dinv, alpha, stop, interior ? max_iter : 0, &it, &rr, s, err))
    return ELM_ERR_CUDA;
  const double rel = bn > 0.0 ? std::sqrt(rr) / bn : std::sqrt(rr);
  if (iters) *iters = it;
  if (resid) *resid = rel;
  if (!chk(cudaMemcpyAsync(c_new, x, bytes, cudaMemcpyDeviceToDevice, s), "result")) return ELM_ERR_CUDA;
  if (!std::isfinite(rel)) {
    *err = "non-finite residual";
    return ELM_ERR_NONFINITE;
  }
  if (rel > rtol && interior) {
    *err = "CG did not reach the tolerance within max_iter iterations (relative residual " + std::to_string(rel) + ")";
    return ELM_ERR_NOT_CONVERGED;
  }
  return ELM_OK;
}

}  // namespace
}  // namespace elm

extern "C" elm_status elm_diffusion_step(elm_mesh me, const void* c_hat_dev, const void* c_bnd_dev,
                                         const void* q_dev, void* c_new_dev, double tau, double kappa, double theta,
                                         double rtol, int max_iter, int* iterations, double* residual,
                                         void* stream) {
  auto fail = [](elm_status st, const std::string& m) {
    elm::set_last_error("elm_diffusion_step: " + m);
    return st;
  };
  if (!me) return fail(ELM_ERR_ARG, "null mesh");
  if (!c_hat_dev || !c_new_dev) return fail(ELM_ERR_ARG, "null buffer");
  if (!std::isfinite(tau) || tau < 0.0 || !std::isfinite(kappa) || kappa < 0.0 || !std::isfinite(theta) ||
      theta < 0.0 || theta > 1.0)
    return fail(ELM_ERR_ARG, "tau, kappa >= 0 finite and theta in [0, 1] required");
  if (!(rtol > 0.0) || max_iter < 0) return fail(ELM_ERR_ARG, "rtol > 0 and max_iter >= 0 required");
  if (me->host_only || !me->with_diffusion)
    return fail(ELM_ERR_STATE, "mesh was created without ELM_DIFFUSION");
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  const size_t bytes = es * size_t(me->n_storage);
  auto overlap = [bytes](const void* a, const void* b) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return a && b && pa < pb + bytes && pb < pa + bytes;
  };
  if (overlap(c_hat_dev, c_new_dev) || overlap(c_bnd_dev, c_new_dev) || overlap(q_dev, c_new_dev))
    return fail(ELM_ERR_ARG, "c_new overlaps an input");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != me->device) cudaSetDevice(me->device);
  std::string err;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  elm_status st = me->precision == ELM_FP64
                      ? (me->blend.nsec > 0
                             ? elm::solve<double>(me, c_hat_dev, c_bnd_dev, q_dev, c_new_dev, tau, kappa, theta, rtol,
                                                  max_iter, iterations, residual, s, &err)
                             : elm::solve_mixed(me, c_hat_dev, c_bnd_dev, q_dev, c_new_dev, tau, kappa, theta, rtol,
                                                max_iter, iterations, residual, s, &err))
                      : elm::solve<float>(me, c_hat_dev, c_bnd_dev, q_dev, c_new_dev, tau, kappa, theta, rtol,
                                          max_iter, iterations, residual, s, &err);
  if (prev >= 0 && prev != me->device) cudaSetDevice(prev);
  return st == ELM_OK ? ELM_OK : fail(st, err);
}
