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
// one stiffness matrix per sigma; a thread per lattice cell applies the
// element matrices of the cell's simplices that lie in the macro.  The
// solver's vectors are in the unique-node layout, so interface nodes shared by
// several macros are single unknowns.
//
// Deterministic assembly without atomics.  Two lattice cells whose indices
// have the same parity in every axis share no node (their node ranges are at
// least one cell apart).  So each of the 2^d parities (colours) has its own
// accumulator vector in the storage layout (each macro writes its own copy of
// an interface node): within one colour every slot has at most one writing
// thread, which stores its cell's sum over the cell's simplices (added in a
// fixed order), and all colours run in one launch.  Colours whose cells do
// not hold a slot leave it zero.  The accumulators are tiled by 32 slots:
// accumulator (slot, colour) sits at ((slot / 32) 2^d + colour) 32 + slot % 32,
// so the 2^d colours of 32 consecutive slots form one contiguous block.  Every
// accumulator that some cell of its colour covers is rewritten by that cell
// on every application (zeros included), and the others are never written
// and stay zero from the set-up.  A fold then adds, for every unique node, its
// storage copies in ascending slot order and, for each copy, the 2^d colour
// values in ascending order.  The summation order is fixed, so results are
// bitwise equal run to run.
//
// Iterations run in batches of kCheckEvery between reads of the residual by
// the host: the scalar kernel sets a done flag on the device once the residual
// (or the iteration budget) is reached, and every later kernel of the batch
// returns at once.
//
// Dirichlet conditions: boundary unknowns keep c_bnd; CG runs on the
// interior unknowns (search directions are zero on the boundary).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
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
// Device: the operator y += scale (M + alpha A) x over all micro simplices.
// ---------------------------------------------------------------------------

// CG scalars on the device.  done: the residual or the iteration budget was
// reached (set by k_cg_scalars); iters: iterations completed.
struct Scalars {
  double rz, rz_new, pq, rr, bb, alpha, beta, stop_rr;
  int done, iters, budget, pad;
};

struct OpArgs {
  const void* tables;       // per macro: M [nb*nb], then A [n_perm][nb*nb]; blended: per simplex
  const int4* chunks;       // work list: (macro, first cell, count, colour) per block
  const int4* cellv;        // cells (c0, c1, c2) of all colours, macro by macro
  const int64_t* unique_map;
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

// ys[colour][slot] = scale (M + alpha A) x summed over the simplices of one
// cell that lie in the macro, for every node of the cell's (P + 1)^d node box,
// into the accumulators of the cell's colour (no two cells of one colour
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
    xc[l] = (!DIAG && ex[l]) ? x[a.unique_map[sl[l]]] : R(0);
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

// y[u] += the sum over the storage copies of unique node u (ascending slot
// order: fold_off / fold_slots) of their NCOL colour accumulators (ascending
// colour; one warp-uniform loop, so every access is coalesced).
template <class R, int NCOL>
__global__ void k_fold(const R* __restrict__ ys, R* __restrict__ y, const int* __restrict__ off,
                       const int* __restrict__ slots, int64_t n, const Scalars* sc) {
  if (sc != nullptr && sc->done) return;
  const int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (u >= n) return;
  R v = R(0);
  for (int k = off[u]; k < off[u + 1]; ++k) {
    const int sl = slots[k];
    const R* e = ys + int64_t(sl >> 5) * (32 * NCOL) + (sl & 31);
    R w[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) w[c] = __ldg(e + 32 * c);
#pragma unroll
    for (int c = 0; c < NCOL; ++c) v += w[c];
  }
  y[u] += v;
}

// ---------------------------------------------------------------------------
// Device: CG vector kernels and deterministic reductions (per-block partials
// in a fixed order, then one block sums the partials in a fixed order).
// ---------------------------------------------------------------------------


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

// r := r with zero boundary; z = dinv r; p = z; q = 0; partials (r.z, r.r).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_start(R* r, R* z, R* p, R* q, const R* dinv, const uint8_t* bnd,
                                                          int64_t n, double* part) {
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
    rz += ri * zi;
    rr += ri * ri;
  }
  const double s1 = block_sum(double(rz), sh);
  __syncthreads();
  const double s2 = block_sum(double(rr), sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

// The CG iteration's operator result and p.q in one pass: q = the fold of
// the colour accumulators (as k_fold; q is overwritten), zero on the
// boundary; partial of p.q.
template <class R, int NCOL>
__global__ void __launch_bounds__(kRedThreads) k_fold_pq(const R* __restrict__ ys, const R* __restrict__ p,
                                                         R* __restrict__ q, const int* __restrict__ off,
                                                         const int* __restrict__ slots, const uint8_t* bnd,
                                                         int64_t n, double* part, const Scalars* sc) {
  __shared__ double sh[kRedThreads / 32];
  if (sc->done) return;
  R pq = R(0);
  for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < n; u += int64_t(gridDim.x) * blockDim.x) {
    R v = R(0);
    for (int k = off[u]; k < off[u + 1]; ++k) {
      const int sl = slots[k];
      const R* e = ys + int64_t(sl >> 5) * (32 * NCOL) + (sl & 31);
      R w[NCOL];
#pragma unroll
      for (int c = 0; c < NCOL; ++c) w[c] = __ldg(e + 32 * c);
#pragma unroll
      for (int c = 0; c < NCOL; ++c) v += w[c];
    }
    if (bnd[u]) v = R(0);
    q[u] = v;
    pq += p[u] * v;
  }
  const double t = block_sum(double(pq), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// x += alpha p; r -= alpha q; z = dinv r; partials (r.z, r.r).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(R* x, R* r, R* z, const R* p, const R* q, const R* dinv,
                                                           const Scalars* sc, int64_t n, double* part) {
  __shared__ double sh[kRedThreads / 32];
  if (sc->done) return;
  const R al = R(sc->alpha);
  R rz = R(0), rr = R(0);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] += al * p[i];
    const R ri = r[i] - al * q[i];
    r[i] = ri;
    const R zi = dinv[i] * ri;
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  const double s1 = block_sum(double(rz), sh);
  __syncthreads();
  const double s2 = block_sum(double(rr), sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[gridDim.x + blockIdx.x] = s2;
  }
}

// p = z + beta p (q is overwritten by the next k_fold_pq).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_cg_direction(R* p, const R* z, const Scalars* sc, int64_t n) {
  if (sc->done) return;
  const R be = R(sc->beta);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z[i] + be * p[i];
}

// Sums the partials of a reduction and updates the CG scalars:
// what = 0: start (rz, rr; the stopping residual and the iteration budget);
// 1: p.q -> alpha; 2: update (rz_new, rr) -> beta, one iteration done.  Sets
// done once |r|^2 <= stop_rr (or it is not finite) or the budget is spent.
__global__ void __launch_bounds__(kRedThreads) k_cg_scalars(const double* part, int nparts, int what, Scalars* sc,
                                                            double stop_rr, int budget) {
  __shared__ double sh[kRedThreads / 32];
  if (what != 0 && sc->done) return;
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    s1 += part[i];
    if (what != 1) s2 += part[nparts + i];
  }
  const double a = block_sum(s1, sh);
  __syncthreads();
  const double b = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    if (what == 0) {
      sc->rz = a;
      sc->rr = b;
      sc->stop_rr = stop_rr;
      sc->budget = budget;
      sc->iters = 0;
      sc->done = (b <= stop_rr || !isfinite(b) || budget <= 0) ? 1 : 0;
    } else if (what == 1) {
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
}

// |b|^2 over the interior unknowns (the residual reference).
template <class R>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const R* b, const uint8_t* bnd, int64_t n, double* part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (!bnd[i]) s += double(b[i]) * double(b[i]);
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

elm_status build_diffusion(elm_mesh_s* me, std::string* err) {
  const int d = me->dim, p = me->order, nb = n_local(d, p), np = n_perm(d);
  const size_t tab = size_t(nb) * nb * (1 + np);
  std::vector<double> t64(tab * me->n_macros);
  for (int64_t m = 0; m < me->n_macros; ++m)
    element_tables(d, p, me->N, me->geo[m], t64.data() + m * tab, t64.data() + m * tab + size_t(nb) * nb);
  // boundary unknowns: a node on face k (barycentric weight k = 0) of a macro
  // whose face k has no neighbour
  std::vector<uint8_t> bnd(me->n_unique, 0);
  {
    const int M = me->M;
    for (int64_t m = 0; m < me->n_macros; ++m) {
      const MacroGeo& g = me->geo[m];
      int64_t slot = m * me->npm;
      int q[3] = {0, 0, 0};
      auto visit = [&]() {
        const int pp[5] = {M, q[0], q[1], d == 3 ? q[2] : 0, 0};
        bool on = false;
        for (int k = 0; k <= d; ++k) {
          const int w = (d == 3 || k < d) ? pp[k] - pp[k + 1] : pp[k];
          if (w == 0 && g.nb[k] < 0) on = true;
        }
        if (on) bnd[me->unique_map[slot]] = 1;
        ++slot;
      };
      if (d == 2) {
        for (q[0] = 0; q[0] <= M; ++q[0])
          for (q[1] = 0; q[1] <= q[0]; ++q[1]) visit();
      } else {
        for (q[0] = 0; q[0] <= M; ++q[0])
          for (q[1] = 0; q[1] <= q[0]; ++q[1])
            for (q[2] = 0; q[2] <= q[1]; ++q[2]) visit();
      }
    }
  }
  // cells of every macro (c0 >= c1 [>= c2] >= 0, c0 < N) by colour (the
  // parity of each index), then macro; chunks of at most kDiffThreads cells
  // of one colour and one macro
  const int ncol = 1 << d;
  std::vector<int4> cells, cellv;
  me->cell_color_off.assign(ncol + 1, 0);
  for (int col = 0; col < ncol; ++col) {
    me->cell_color_off[col] = int64_t(cells.size());
    for (int64_t m = 0; m < me->n_macros; ++m) {
      const int64_t first = int64_t(cellv.size());
      for (int c0 = col & 1; c0 < me->N; c0 += 2)
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
  }
  me->cell_color_off[ncol] = int64_t(cells.size());
  me->n_cell_chunks = int64_t(cells.size());
  // fold lists: the storage copies of every unique node in ascending slot order
  std::vector<int> foff(me->n_unique + 1, 0), fslots(me->n_storage);
  for (int64_t sl = 0; sl < me->n_storage; ++sl) ++foff[me->unique_map[sl] + 1];
  for (int64_t u = 0; u < me->n_unique; ++u) foff[u + 1] += foff[u];
  {
    std::vector<int> next(foff.begin(), foff.end() - 1);
    for (int64_t sl = 0; sl < me->n_storage; ++sl) fslots[next[me->unique_map[sl]]++] = int(sl);
  }
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  bool ok = true;
  ok = ok && cudaMalloc(&me->d_dtab, tab * me->n_macros * es) == cudaSuccess;
  if (ok) {
    if (me->precision == ELM_FP64) {
      ok = cudaMemcpy(me->d_dtab, t64.data(), tab * me->n_macros * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
      std::vector<float> t32(t64.begin(), t64.end());
      ok = cudaMemcpy(me->d_dtab, t32.data(), tab * me->n_macros * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  ok = ok && cudaMalloc((void**)&me->d_dbnd, me->n_unique) == cudaSuccess &&
       cudaMemcpy(me->d_dbnd, bnd.data(), me->n_unique, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dcells, sizeof(int4) * cells.size()) == cudaSuccess &&
       cudaMemcpy(me->d_dcells, cells.data(), sizeof(int4) * cells.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dcellv, sizeof(int4) * cellv.size()) == cudaSuccess &&
       cudaMemcpy(me->d_dcellv, cellv.data(), sizeof(int4) * cellv.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dfold_off, sizeof(int) * foff.size()) == cudaSuccess &&
       cudaMemcpy(me->d_dfold_off, foff.data(), sizeof(int) * foff.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dfold_slots, sizeof(int) * fslots.size()) == cudaSuccess &&
       cudaMemcpy(me->d_dfold_slots, fslots.data(), sizeof(int) * fslots.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  // the colour accumulators, tiled by 32 slots, in the mesh precision (and a
  // second, FP32 set for the inner solves of FP64 meshes: the zero entries no
  // cell writes must stay zero in each precision's own layout); zero where no
  // cell of the colour ever writes
  const size_t ysn = size_t((me->n_storage + 31) / 32 * 32) * size_t(ncol);
  ok = ok && cudaMalloc(&me->d_dys, ysn * es) == cudaSuccess && cudaMemset(me->d_dys, 0, ysn * es) == cudaSuccess;
  if (me->precision == ELM_FP64)
    ok = ok && cudaMalloc(&me->d_dys32, ysn * 4) == cudaSuccess && cudaMemset(me->d_dys32, 0, ysn * 4) == cudaSuccess;
  ok = ok && cudaMalloc(&me->d_dvec, size_t(kDiffVectors) * me->n_unique * es) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dpart, sizeof(double) * 2 * kRedMaxBlocks) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&me->d_dscal, sizeof(Scalars) + 2 * sizeof(double)) == cudaSuccess;
  if (me->precision == ELM_FP64) {
    // FP32 copies for the inner solves of the mixed-precision form
    std::vector<float> t32(t64.begin(), t64.end());
    ok = ok && cudaMalloc(&me->d_dtab32, tab * me->n_macros * 4) == cudaSuccess &&
         cudaMemcpy(me->d_dtab32, t32.data(), tab * me->n_macros * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMalloc(&me->d_dvec32, size_t(kDiffVectors32) * me->n_unique * 4) == cudaSuccess;
  }
  if (!ok) {
    *err = std::string("diffusion tables: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  me->n_boundary = 0;
  for (uint8_t b : bnd) me->n_boundary += b;
  return ELM_OK;
}

elm_status build_diffusion_blended(elm_mesh_s* me, std::string* err) {
  std::vector<double> t;
  blended_element_tables(me, t);
  cudaFree(me->d_dtab_el);
  me->d_dtab_el = nullptr;
  if (cudaMalloc(&me->d_dtab_el, t.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(me->d_dtab_el, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = std::string("blended diffusion tables: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  return ELM_OK;
}

namespace {

// y += scale (M + alpha A) x (diag: the diagonal only): the cell pass into
// the colour accumulators, then (fold) their fold into y.  tables: the element
// tables in the precision R (null: the mesh's own).  sc: the CG scalars whose
// done flag ends the work early (null: always applied).
template <class R>
cudaError_t apply_op(const elm_mesh_s* me, const R* x, R* y, double alpha, double scale, bool diag, cudaStream_t s,
                     const void* tables = nullptr, const Scalars* sc = nullptr, bool fold = true) {
  const bool blended = me->blend.nsec > 0;
  OpArgs a{tables ? tables : (blended ? me->d_dtab_el : me->d_dtab), me->d_dcells, me->d_dcellv, me->d_unique_map,
           int(me->npm), me->N, sc};
  R* ys = static_cast<R*>(sizeof(R) == 4 && me->precision == ELM_FP64 ? me->d_dys32 : me->d_dys);
  const R al = R(alpha), sca = R(scale);
  const unsigned g = unsigned(me->n_cell_chunks);
  if (g > 0) {
    bool launched = false;
    if constexpr (sizeof(R) == 8) {
      if (blended) {  // 2D FP64 only (elm_mesh_set_annulus)
        if (me->order == 2) {
          if (diag) k_apply<2, R, 2, true, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
          else k_apply<2, R, 2, false, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
        } else {
          if (diag) k_apply<2, R, 1, true, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
          else k_apply<2, R, 1, false, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
        }
        launched = true;
      }
    }
    if (!launched) {
      if (blended) return cudaErrorInvalidValue;
#define ELM_APPLY(DD, PP)                                                              \
  if (diag) k_apply<DD, R, PP, true><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);   \
  else k_apply<DD, R, PP, false><<<g, kDiffThreads, 0, s>>>(a, x, ys, al, sca);
      if (me->dim == 3) {
        if (me->order == 2) { ELM_APPLY(3, 2) } else { ELM_APPLY(3, 1) }
      } else {
        if (me->order == 2) { ELM_APPLY(2, 2) } else { ELM_APPLY(2, 1) }
      }
#undef ELM_APPLY
    }
  }
  const int64_t n = me->n_unique;
  const unsigned fb = unsigned((n + 255) / 256);
  if (fold && n > 0) {
    if (me->dim == 3)
      k_fold<R, 8><<<fb, 256, 0, s>>>(ys, y, me->d_dfold_off, me->d_dfold_slots, n, sc);
    else
      k_fold<R, 4><<<fb, 256, 0, s>>>(ys, y, me->d_dfold_off, me->d_dfold_slots, n, sc);
  }
  return cudaGetLastError();
}

// PCG iterations on the interior from the state of k_cg_start (r, z = D^{-1} r,
// p = z; its partials of r.z and r.r in the reduction space): stops when
// |r|^2 <= stop_rr or after `budget` iterations.  The iterations are enqueued
// in batches of kCheckEvery; the device sets the done flag (k_cg_scalars) and
// the kernels after it return at once, so the host reads the scalars once per
// batch.  *done = iterations run, *rr = final |r|^2.  Returns false on a CUDA
// error (message in *err).
constexpr int kCheckEvery = 8;

template <class R>
bool pcg_iterate(const elm_mesh_s* me, const void* tab, R* x, R* r, R* z, R* p, R* qv, const R* dinv, double alpha,
                 double stop_rr, int budget, int* done, double* rr, cudaStream_t s, std::string* err) {
  const int64_t n = me->n_unique;
  double* part = me->d_dpart;
  Scalars* sc = reinterpret_cast<Scalars*>(me->d_dscal);
  const int nred = red_blocks(n);
  auto chk = [&](cudaError_t e, const char* where) {
    if (e != cudaSuccess) *err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  k_cg_scalars<<<1, kRedThreads, 0, s>>>(part, nred, 0, sc, stop_rr, budget);
  Scalars h{};
  for (;;) {
    if (!chk(cudaMemcpyAsync(&h, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s), "read") ||
        !chk(cudaStreamSynchronize(s), "sync"))
      return false;
    if (h.done) break;
    for (int k = 0; k < kCheckEvery; ++k) {
      // q = E p (the fold of the cell pass) and p.q in one pass
      if (!chk(apply_op<R>(me, p, qv, alpha, 1.0, false, s, tab, sc, false), "apply")) return false;
      const R* ys = static_cast<const R*>(sizeof(R) == 4 && me->precision == ELM_FP64 ? me->d_dys32 : me->d_dys);
      if (me->dim == 3)
        k_fold_pq<R, 8><<<nred, kRedThreads, 0, s>>>(ys, p, qv, me->d_dfold_off, me->d_dfold_slots, me->d_dbnd, n,
                                                     part, sc);
      else
        k_fold_pq<R, 4><<<nred, kRedThreads, 0, s>>>(ys, p, qv, me->d_dfold_off, me->d_dfold_slots, me->d_dbnd, n,
                                                     part, sc);
      k_cg_scalars<<<1, kRedThreads, 0, s>>>(part, nred, 1, sc, 0.0, 0);
      k_cg_update<R><<<nred, kRedThreads, 0, s>>>(x, r, z, p, qv, dinv, sc, n, part);
      k_cg_scalars<<<1, kRedThreads, 0, s>>>(part, nred, 2, sc, 0.0, 0);
      k_cg_direction<R><<<nred, kRedThreads, 0, s>>>(p, z, sc, n);
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
// applications instead of one per iteration: the FP64 element products run on
// this part's narrow FP64 pipe, the FP32 ones on its FP32 pipe.
constexpr double kInnerRtol = 3e-5;

elm_status solve_mixed(elm_mesh_s* me, const void* c_hat, const void* c_bnd, const void* q, void* c_new,
                       double tau, double kappa, double theta, double rtol, int max_iter, int* iters, double* resid,
                       cudaStream_t s, std::string* err) {
  const int64_t n = me->n_unique;
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
  if (!chk(launch_gather(ELM_FP64, c_hat, x, me->d_owner, n, 1, s), "gather c_hat")) return ELM_ERR_CUDA;
  if (!chk(cudaMemsetAsync(b, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<double>(me, x, b, -tau * (1.0 - theta) * kappa, 1.0, false, s), "rhs")) return ELM_ERR_CUDA;
  if (q) {
    if (!chk(launch_gather(ELM_FP64, q, tmp, me->d_owner, n, 1, s), "gather q")) return ELM_ERR_CUDA;
    if (!chk(apply_op<double>(me, tmp, b, 0.0, tau, false, s), "source")) return ELM_ERR_CUDA;
  }
  if (c_bnd) {
    if (!chk(launch_gather(ELM_FP64, c_bnd, tmp, me->d_owner, n, 1, s), "gather c_bnd")) return ELM_ERR_CUDA;
    k_set_boundary<double><<<eb, 256, 0, s>>>(x, tmp, me->d_dbnd, n);
  }
  const double alpha = tau * theta * kappa;
  if (!chk(cudaMemsetAsync(dinv32, 0, size_t(n) * 4, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<float>(me, nullptr, dinv32, alpha, 1.0, true, s, me->d_dtab32), "diagonal")) return ELM_ERR_CUDA;
  k_invert_diag<float><<<eb, 256, 0, s>>>(dinv32, me->d_dbnd, n);
  k_norm2<double><<<nred, kRedThreads, 0, s>>>(b, me->d_dbnd, n, part);
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
    k_norm2<double><<<nred, kRedThreads, 0, s>>>(r, me->d_dbnd, n, part);
    k_sum_into<<<1, kRedThreads, 0, s>>>(part, nred, rnorm);
    double hr = 0.0;
    if (!chk(cudaMemcpyAsync(&hr, rnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "read") ||
        !chk(cudaStreamSynchronize(s), "sync"))
      return ELM_ERR_CUDA;
    rel = bn > 0.0 ? std::sqrt(hr) / bn : std::sqrt(hr);
    if (!interior || !(rel > rtol) || total >= max_iter || !std::isfinite(rel)) break;
    // inner FP32 solve of E d = r from d = 0
    k_residual_to_float<<<eb, 256, 0, s>>>(r, r32, d32, me->d_dbnd, n);
    k_cg_start<float><<<nred, kRedThreads, 0, s>>>(r32, z32, p32, q32, dinv32, me->d_dbnd, n, part);
    int done = 0;
    double rr32 = 0.0;
    // stop at kInnerRtol of the inner start, or where the outer tolerance is met
    const double start_rr = hr;
    const double stop = std::max(kInnerRtol * kInnerRtol * start_rr, 0.25 * rtol * rtol * bn * bn);
    if (!pcg_iterate<float>(me, me->d_dtab32, d32, r32, z32, p32, q32, dinv32, alpha, stop, max_iter - total,
                            &done, &rr32, s, err))
      return ELM_ERR_CUDA;
    total += done;
    k_add_correction<<<eb, 256, 0, s>>>(x, d32, n);
    if (outer > 64) break;  // safeguard: corrections stopped converging
  }
  if (iters) *iters = total;
  if (resid) *resid = rel;
  if (!chk(launch_gather(ELM_FP64, x, c_new, me->d_unique_map, me->n_storage, 1, s), "scatter")) return ELM_ERR_CUDA;
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
  const int64_t n = me->n_unique;
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
  // c_hat (storage) -> x (unique); right-hand side b
  if (!chk(launch_gather(prec, c_hat, x, me->d_owner, n, 1, s), "gather c_hat")) return ELM_ERR_CUDA;
  if (!chk(cudaMemsetAsync(b, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<R>(me, x, b, -tau * (1.0 - theta) * kappa, 1.0, false, s), "rhs")) return ELM_ERR_CUDA;
  if (q) {
    if (!chk(launch_gather(prec, q, z, me->d_owner, n, 1, s), "gather q")) return ELM_ERR_CUDA;
    if (!chk(apply_op<R>(me, z, b, 0.0, tau, false, s), "source")) return ELM_ERR_CUDA;
  }
  if (c_bnd) {
    if (!chk(launch_gather(prec, c_bnd, z, me->d_owner, n, 1, s), "gather c_bnd")) return ELM_ERR_CUDA;
    k_set_boundary<R><<<eb, 256, 0, s>>>(x, z, me->d_dbnd, n);
  }
  // Jacobi preconditioner of E = M + tau theta kappa A
  const double alpha = tau * theta * kappa;
  if (!chk(cudaMemsetAsync(dinv, 0, bytes, s), "memset")) return ELM_ERR_CUDA;
  if (!chk(apply_op<R>(me, x, dinv, alpha, 1.0, true, s), "diagonal")) return ELM_ERR_CUDA;
  k_invert_diag<R><<<eb, 256, 0, s>>>(dinv, me->d_dbnd, n);
  k_norm2<R><<<nred, kRedThreads, 0, s>>>(b, me->d_dbnd, n, part);
  k_sum_into<<<1, kRedThreads, 0, s>>>(part, nred, bnorm);
  // r = b - E x, restricted to the interior; z = D^{-1} r; p = z
  k_copy<R><<<eb, 256, 0, s>>>(r, b, n);
  if (!chk(apply_op<R>(me, x, r, alpha, -1.0, false, s), "residual")) return ELM_ERR_CUDA;
  k_cg_start<R><<<nred, kRedThreads, 0, s>>>(r, z, p, qv, dinv, me->d_dbnd, n, part);
  double hb = 0.0;
  if (!chk(cudaMemcpyAsync(&hb, bnorm, sizeof(double), cudaMemcpyDeviceToHost, s), "read") ||
      !chk(cudaStreamSynchronize(s), "sync"))
    return ELM_ERR_CUDA;
  const double bn = std::sqrt(hb);
  const bool interior = me->n_unique > me->n_boundary;
  int it = 0;
  double rr = 0.0;
  const double stop = bn > 0.0 ? rtol * rtol * bn * bn : rtol * rtol;
  if (!pcg_iterate<R>(me, nullptr, x, r, z, p, qv, dinv, alpha, stop, interior ? max_iter : 0, &it, &rr, s, err))
    return ELM_ERR_CUDA;
  const double rel = bn > 0.0 ? std::sqrt(rr) / bn : std::sqrt(rr);
  if (iters) *iters = it;
  if (resid) *resid = rel;
  if (!chk(launch_gather(prec, x, c_new, me->d_unique_map, me->n_storage, 1, s), "scatter")) return ELM_ERR_CUDA;
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
