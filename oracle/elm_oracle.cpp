// elm_oracle.cpp -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
//
// A slow, plain, FP64 CPU restatement of the advection step of the modified
// method of characteristics (MMOC) of Kohl, Mohr, Eibl and Ruede (arXiv
// 2103.02388).  Only tests/, the smoke check and the CPU-baseline leg of the
// benchmark may load this library.  It shares no code, header, table or helper
// with the CUDA library; the only thing the two sides have in common is the
// seeded input arrays the tests hand to both.
//
// What it computes, step by step, in the order of the paper:
//   * Sec. 2.1 (hierarchical hybrid grids): a coarse mesh of macro triangles or
//     tetrahedra, each refined uniformly (Bey) L times.  For a simplex whose
//     vertices are taken in ascending global id order this refinement is the
//     Freudenthal/Kuhn subdivision of the reference simplex
//     {N >= q1 >= q2 >= q3 >= 0}, N = 2^L.
//   * Sec. 2.2 (spaces S^m_l) and Sec. 3.1 (linear or quadratic Lagrange
//     elements): P2 nodes = micro vertices and edge midpoints, P1 nodes = micro
//     vertices; a global node is identified by the macro vertices it lies
//     between and its integer barycentric weights, so nodes shared by several
//     macros are one unknown.
//   * Eq. (characteristic curves) / Eq. (departure point): X(x, t_{n+1}, t_n)
//     integrated backwards with classic RK4 (Sec. 3.1 "Test setup"), with
//     n_sub equal substeps.
//   * Eq. (linear interpolation): the velocity at a stage time is the linear
//     time interpolant of u^n_h and u^{n+1}_h.
//   * Sec. 2.3.2, field evaluation: locate the macro (here: brute force over all
//     macros, keeping the one with the largest minimum barycentric), locate the
//     micro element in O(1) (floor + sort of the fractional parts), pull back to
//     the micro element (solve its barycentric system) and sum the P1 or P2
//     basis.
//   * Step (iii): T^{n+1}_i = c^n_h(X_i) (kappa = 0, no diffusion).
//   * Sec. 3.1: the error metrics need e^T M e with the P1 / P2 mass matrix M,
//     assembled here element by element from exact barycentric-monomial
//     integrals.
//   * Sec. 2.3.3 (look-back distance): a trace continued from given points
//     over a further time interval with that interval's velocity pair, so a
//     trace can span several time steps (b > 1) before T is evaluated.
//   * Eq. (departure point), differentiated: forward-mode (dual number)
//     directional derivatives of T^{n+1} with respect to the nodal velocity and
//     the transpose of the interpolation for T^n, used to check adjoints.
//
// Readings of points the paper leaves open:
//   * Out-of-domain stage points: every RK stage point and the final departure
//     point are clamped componentwise to the axis-aligned bounding box of the
//     mesh (the Euclidean projection for box domains).  If the clamped point
//     still lies outside every macro (non-box domains only), its barycentric
//     coordinates in the closest macro are clamped at 0 and renormalised.
//   * Micro-face ties: floor, cell clamped to [0, N-1], ties in the sort broken
//     by axis index; any containing element is valid because P2 is C0.
//   * Steady velocity (u_old and u_new the same array): no time interpolation.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -pthread elm_oracle.cpp -o liboracle.so

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Small dense linear algebra (Gauss-Jordan with partial pivoting).
// ---------------------------------------------------------------------------

// Solves A z = b for an n x n system (n <= 4), row-major A.  Returns false if
// the matrix is singular.
bool solve_small(int n, const double* A_in, const double* b_in, double* z) {
  double A[4][5];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[i][j] = A_in[i * n + j];
    A[i][n] = b_in[i];
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return false;
    if (piv != col)
      for (int j = 0; j <= n; ++j) std::swap(A[piv][j], A[col][j]);
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = A[r][col] / A[col][col];
      for (int j = col; j <= n; ++j) A[r][j] -= f * A[col][j];
    }
  }
  for (int i = 0; i < n; ++i) z[i] = A[i][n] / A[i][i];
  return true;
}

// Barycentric coordinates of point y with respect to the simplex with
// vertices V[0..d] (each d coordinates): solve [V_0 .. V_d ; 1 .. 1] lam = [y; 1].
bool barycentric(int d, const double V[4][3], const double* y, double* lam) {
  double A[16], b[4];
  const int n = d + 1;
  for (int r = 0; r < d; ++r) {
    for (int c = 0; c < n; ++c) A[r * n + c] = V[c][r];
    b[r] = y[r];
  }
  for (int c = 0; c < n; ++c) A[d * n + c] = 1.0;
  b[d] = 1.0;
  return solve_small(n, A, b, lam);
}

// ---------------------------------------------------------------------------
// Mesh: macro simplices, uniform refinement, P1 / P2 node numbering (Sec. 2.1,
// 2.2).
// ---------------------------------------------------------------------------

struct Macro {
  int64_t v[4];      // global vertex ids in ascending order (Kuhn order)
  double P[4][3];    // their coordinates
};

// Blending (Sec. 2.1, blending map Phi): a 2D macro mesh that is a ring of
// n sectors between two regular n-gons, with vertices on the circles r_min and
// r_max at the angles theta_k = theta0 + k Delta, Delta = 2 pi / n, is mapped
// onto the annulus sector by sector in polar form: a computational point
// x = rho ((1 - lam) e_k + lam e_{k+1}) (e_k the unit vector at theta_k, rho
// running from r_min on the inner chord to r_max on the outer one) goes to
// rho e(theta_k + lam Delta).  Vertices stay, chords become arcs with uniform
// angle along them, and det DPhi = Delta / sin(Delta) everywhere.
struct Blend {
  bool on = false;
  double rmin = 0.0, rmax = 0.0, theta0 = 0.0;
  int nsec = 0;
};

struct Mesh {
  int d = 0, L = 0, N = 0, M = 0;   // dimension, level, N = 2^L, M = order * N
  int order = 2;                     // 1: P1 (nodes = micro vertices), 2: P2
  std::vector<Macro> mac;
  std::vector<std::vector<int32_t>> id;  // per macro: dense (M+1)^d table p -> node
  std::vector<double> X;                 // node coordinates, [n_nodes, d] (physical: Phi applied)
  Blend bl;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int64_t n_nodes = 0;

  int64_t dense(const int* p) const {
    int64_t k = 0;
    for (int i = 0; i < d; ++i) k = k * (M + 1) + p[i];
    return k;
  }
};

// Barycentric integer weights of the lattice point p (M >= p1 >= ... >= pd >= 0)
// of the reference Kuhn simplex: w_k = p_k - p_{k+1} with p_0 = M, p_{d+1} = 0.
void lattice_weights(int d, int M, const int* p, int* w) {
  int pp[5];
  pp[0] = M;
  for (int i = 0; i < d; ++i) pp[i + 1] = p[i];
  pp[d + 1] = 0;
  for (int k = 0; k <= d; ++k) w[k] = pp[k] - pp[k + 1];
}

// Physical position of a lattice point with weights w (sum = den).
void lattice_point(const Macro& m, int d, const int* w, int den, double* x) {
  for (int r = 0; r < d; ++r) {
    double s = 0.0;
    for (int k = 0; k <= d; ++k) s += double(w[k]) * m.P[k][r];
    x[r] = s / double(den);
  }
}

// Calls f(p) for every lattice point of the reference simplex with side M.
template <class F>
void for_each_lattice_point(int d, int M, F&& f) {
  int p[3] = {0, 0, 0};
  if (d == 2) {
    for (p[0] = 0; p[0] <= M; ++p[0])
      for (p[1] = 0; p[1] <= p[0]; ++p[1]) f(p);
  } else {
    for (p[0] = 0; p[0] <= M; ++p[0])
      for (p[1] = 0; p[1] <= p[0]; ++p[1])
        for (p[2] = 0; p[2] <= p[1]; ++p[2]) f(p);
  }
}

Mesh* build_mesh(int d, int64_t nv, const double* xyz, int64_t nm, const int64_t* mv, int level, int order) {
  if ((d != 2 && d != 3) || nv <= 0 || nm <= 0 || level < 0 || (order != 1 && order != 2)) return nullptr;
  // dense per-macro node tables of (M + 1)^d entries: M <= 1024 (2D), 256 (3D)
  if (level > 12 || (order << level) > (d == 2 ? 1024 : 256)) return nullptr;
  Mesh* me = new Mesh();
  me->d = d;
  me->L = level;
  me->order = order;
  me->N = 1 << level;
  me->M = order * me->N;
  for (int r = 0; r < d; ++r) {
    me->lo[r] = std::numeric_limits<double>::infinity();
    me->hi[r] = -std::numeric_limits<double>::infinity();
  }
  for (int64_t i = 0; i < nv; ++i)
    for (int r = 0; r < d; ++r) {
      me->lo[r] = std::min(me->lo[r], xyz[i * d + r]);
      me->hi[r] = std::max(me->hi[r], xyz[i * d + r]);
    }
  me->mac.resize(nm);
  for (int64_t m = 0; m < nm; ++m) {
    Macro& mc = me->mac[m];
    for (int k = 0; k <= d; ++k) mc.v[k] = mv[m * (d + 1) + k];
    std::sort(mc.v, mc.v + d + 1);
    for (int k = 0; k <= d; ++k) {
      if (mc.v[k] < 0 || mc.v[k] >= nv) { delete me; return nullptr; }
      for (int r = 0; r < d; ++r) mc.P[k][r] = xyz[mc.v[k] * d + r];
    }
  }
  // Global node numbering.  Interior lattice points (all weights > 0) belong
  // to one macro only; points on a macro face, edge or vertex are keyed by the
  // (vertex id, weight) pairs with non-zero weight so that all macros sharing
  // them agree on one node.
  const int M = me->M;
  int64_t per_macro = 1;
  for (int i = 0; i < d; ++i) per_macro *= (M + 1);
  me->id.assign(nm, std::vector<int32_t>(per_macro, -1));
  std::map<std::vector<int64_t>, int32_t> shared;
  int64_t next = 0;
  std::vector<double>& X = me->X;
  for (int64_t m = 0; m < nm; ++m) {
    const Macro& mc = me->mac[m];
    for_each_lattice_point(d, M, [&](const int* p) {
      int w[4];
      lattice_weights(d, M, p, w);
      bool interior = true;
      for (int k = 0; k <= d; ++k) interior = interior && (w[k] > 0);
      int32_t nid;
      if (interior) {
        nid = int32_t(next++);
      } else {
        std::vector<int64_t> key;
        for (int k = 0; k <= d; ++k)
          if (w[k] > 0) { key.push_back(mc.v[k]); key.push_back(w[k]); }
        auto it = shared.find(key);
        if (it != shared.end()) {
          me->id[m][me->dense(p)] = it->second;
          return;
        }
        nid = int32_t(next++);
        shared.emplace(std::move(key), nid);
      }
      me->id[m][me->dense(p)] = nid;
      double x[3];
      lattice_point(mc, d, w, M, x);
      for (int r = 0; r < d; ++r) X.push_back(x[r]);
    });
  }
  me->n_nodes = next;
  return me;
}

// ---------------------------------------------------------------------------
// Field evaluation (Sec. 2.3.2, field evaluation).
// ---------------------------------------------------------------------------

struct Located {
  int64_t macro;
  int w[4][3];      // micro vertices as lattice points of the level-L grid (q space)
  double mu[4];     // barycentric coordinates of the point in that micro simplex
};

// Sector k of the polar angle of x (x != 0) and lam = (theta - theta_k)/Delta.
void blend_sector(const Blend& b, double theta, int* k, double* lam) {
  const double pi = 3.14159265358979323846;
  const double delta = 2.0 * pi / b.nsec;
  const double t = (theta - b.theta0) / delta;
  double kf = std::floor(t);
  *lam = t - kf;
  int kk = int(kf) % b.nsec;
  if (kk < 0) kk += b.nsec;
  *k = kk;
}

void blend_phi(const Blend& b, const double* xc, double* xp) {
  const double pi = 3.14159265358979323846;
  const double delta = 2.0 * pi / b.nsec;
  int k;
  double lam0;
  blend_sector(b, std::atan2(xc[1], xc[0]), &k, &lam0);
  const double tk = b.theta0 + k * delta, tk1 = tk + delta;
  const double ek[2] = {std::cos(tk), std::sin(tk)}, ek1[2] = {std::cos(tk1), std::sin(tk1)};
  // x parallel to p(lam) = (1 - lam) e_k + lam e_{k+1}
  const double ck = ek[0] * xc[1] - ek[1] * xc[0], ck1 = ek1[0] * xc[1] - ek1[1] * xc[0];
  const double lam = ck / (ck - ck1);
  const double p[2] = {(1 - lam) * ek[0] + lam * ek1[0], (1 - lam) * ek[1] + lam * ek1[1]};
  const double rho = std::sqrt(xc[0] * xc[0] + xc[1] * xc[1]) / std::sqrt(p[0] * p[0] + p[1] * p[1]);
  const double th = tk + lam * delta;
  xp[0] = rho * std::cos(th);
  xp[1] = rho * std::sin(th);
}

void blend_phi_inv(const Blend& b, const double* xp, double* xc) {
  const double pi = 3.14159265358979323846;
  const double delta = 2.0 * pi / b.nsec;
  int k;
  double lam;
  blend_sector(b, std::atan2(xp[1], xp[0]), &k, &lam);
  const double tk = b.theta0 + k * delta, tk1 = tk + delta;
  const double rho = std::sqrt(xp[0] * xp[0] + xp[1] * xp[1]);
  xc[0] = rho * ((1 - lam) * std::cos(tk) + lam * std::cos(tk1));
  xc[1] = rho * ((1 - lam) * std::sin(tk) + lam * std::sin(tk1));
}

// Domain rule for points outside the domain: componentwise clamp to the
// bounding box (box domains: the Euclidean projection); on a blended annulus
// the radius is clamped to [r_min, r_max] (its Euclidean projection).
void clamp_to_box(const Mesh& me, double* y) {
  if (me.bl.on) {
    const double r = std::sqrt(y[0] * y[0] + y[1] * y[1]);
    if (r == 0.0) {
      y[0] = me.bl.rmin;
      y[1] = 0.0;
    } else if (r < me.bl.rmin || r > me.bl.rmax) {
      const double t = std::min(std::max(r, me.bl.rmin), me.bl.rmax) / r;
      y[0] *= t;
      y[1] *= t;
    }
    return;
  }
  for (int r = 0; r < me.d; ++r) y[r] = std::min(std::max(y[r], me.lo[r]), me.hi[r]);
}

// Locates y (already clamped to the box).  May move y onto the mesh boundary
// when y is outside every macro (non-box domains).
void locate(const Mesh& me, double* y, Located& out) {
  const int d = me.d;
  // Macro: brute force, keep the macro with the largest minimum barycentric.
  int64_t best = -1;
  double best_min = -std::numeric_limits<double>::infinity();
  double lam_best[4] = {0, 0, 0, 0};
  for (int64_t m = 0; m < (int64_t)me.mac.size(); ++m) {
    double lam[4];
    if (!barycentric(d, me.mac[m].P, y, lam)) continue;
    double mn = lam[0];
    for (int k = 1; k <= d; ++k) mn = std::min(mn, lam[k]);
    if (mn > best_min) {
      best_min = mn;
      best = m;
      std::memcpy(lam_best, lam, sizeof(lam));
    }
  }
  const Macro& mc = me.mac[best];
  if (best_min < -1e-12) {
    // Outside the mesh: clamp the barycentric coordinates at zero and renormalise.
    double s = 0.0;
    for (int k = 0; k <= d; ++k) { lam_best[k] = std::max(lam_best[k], 0.0); s += lam_best[k]; }
    for (int k = 0; k <= d; ++k) lam_best[k] /= s;
    for (int r = 0; r < d; ++r) {
      double v = 0.0;
      for (int k = 0; k <= d; ++k) v += lam_best[k] * mc.P[k][r];
      y[r] = v;
    }
  }
  out.macro = best;
  // Reference Kuhn coordinates: s_k = lam_k + ... + lam_d (k = 1..d); q = N s.
  double q[3];
  for (int k = 1; k <= d; ++k) {
    double s = 0.0;
    for (int j = k; j <= d; ++j) s += lam_best[j];
    q[k - 1] = me.N * s;
  }
  // Keep q in the closed reference simplex N >= q1 >= ... >= qd >= 0 (this only
  // moves points that are outside by rounding).
  q[0] = std::min(std::max(q[0], 0.0), double(me.N));
  for (int k = 1; k < d; ++k) q[k] = std::min(std::max(q[k], 0.0), q[k - 1]);
  // Micro element in O(1): cell = floor(q) clamped to [0, N-1]; the Kuhn
  // simplex of the cell is fixed by the descending order of the fractions.
  int c[3];
  double f[3];
  for (int k = 0; k < d; ++k) {
    c[k] = std::min(int(std::floor(q[k])), me.N - 1);
    f[k] = q[k] - c[k];
  }
  int order[3] = {0, 1, 2};
  std::stable_sort(order, order + d, [&](int a, int b) { return f[a] > f[b]; });
  for (int r = 0; r < d; ++r) out.w[0][r] = c[r];
  for (int j = 1; j <= d; ++j) {
    for (int r = 0; r < d; ++r) out.w[j][r] = out.w[j - 1][r];
    out.w[j][order[j - 1]] += 1;
  }
  // Pull back: barycentric coordinates in the physical micro simplex.
  double V[4][3];
  for (int j = 0; j <= d; ++j) {
    int wt[4];
    lattice_weights(d, me.N, out.w[j], wt);
    lattice_point(mc, d, wt, me.N, V[j]);
  }
  barycentric(d, V, y, out.mu);
}

// The (d+1)(d+2)/2 P2 nodes of a located micro simplex with their basis values:
// vertex v -> mu_v (2 mu_v - 1); edge (a, b) -> 4 mu_a mu_b  (Sec. 2.2, P2).
int p2_stencil(const Mesh& me, const Located& lc, int32_t* node, double* phi) {
  if (me.order != 2) return 0;
  const int d = me.d;
  int n = 0;
  for (int v = 0; v <= d; ++v) {
    int p[3];
    for (int r = 0; r < d; ++r) p[r] = 2 * lc.w[v][r];
    node[n] = me.id[lc.macro][me.dense(p)];
    phi[n] = lc.mu[v] * (2.0 * lc.mu[v] - 1.0);
    ++n;
  }
  for (int a = 0; a <= d; ++a)
    for (int b = a + 1; b <= d; ++b) {
      int p[3];
      for (int r = 0; r < d; ++r) p[r] = lc.w[a][r] + lc.w[b][r];
      node[n] = me.id[lc.macro][me.dense(p)];
      phi[n] = 4.0 * lc.mu[a] * lc.mu[b];
      ++n;
    }
  return n;
}

// The d+1 P1 nodes of a located micro simplex (its vertices, lattice = the
// level-L grid) with their basis values mu_v (Sec. 3.1, linear elements).
int p1_stencil(const Mesh& me, const Located& lc, int32_t* node, double* phi) {
  if (me.order != 1) return 0;
  for (int v = 0; v <= me.d; ++v) {
    node[v] = me.id[lc.macro][me.dense(lc.w[v])];
    phi[v] = lc.mu[v];
  }
  return me.d + 1;
}

int stencil(const Mesh& me, const Located& lc, int32_t* node, double* phi) {
  return me.order == 1 ? p1_stencil(me, lc, node, phi) : p2_stencil(me, lc, node, phi);
}

// Evaluates an ncomp-component P1 / P2 field (node-major [n_nodes, ncomp]) at y
// (physical; pulled back with Phi^{-1} on a blended mesh).
void eval_field(const Mesh& me, const double* F, int ncomp, double* y, double* out) {
  Located lc;
  double yc[3] = {y[0], y[1], me.d == 3 ? y[2] : 0.0};
  if (me.bl.on) blend_phi_inv(me.bl, y, yc);
  locate(me, yc, lc);
  int32_t node[10];
  double phi[10];
  int n = stencil(me, lc, node, phi);
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += phi[j] * F[int64_t(node[j]) * ncomp + c];
    out[c] = s;
  }
}

// ---------------------------------------------------------------------------
// Departure points: Eq. (departure point) by classic RK4 backwards in time,
// velocity interpolated linearly in time, Eq. (linear interpolation).
// ---------------------------------------------------------------------------

struct Velocity {
  const double* u_old;   // u^n_h   at t_n
  const double* u_new;   // u^{n+1}_h at t_{n+1}
  double dt;
};

// u~(y) at the stage time t~ = t_{n+1} - back, back in [0, dt]:
// (t_{n+1} - t~)/dt * u^n + (t~ - t_n)/dt * u^{n+1}.
void velocity_at(const Mesh& me, const Velocity& V, double back, double* y, double* k) {
  const int d = me.d;
  double a[3], b[3];
  eval_field(me, V.u_new, d, y, b);
  if (V.u_old == V.u_new) {
    for (int r = 0; r < d; ++r) k[r] = b[r];
    return;
  }
  eval_field(me, V.u_old, d, y, a);
  const double w_old = back / V.dt, w_new = (V.dt - back) / V.dt;
  for (int r = 0; r < d; ++r) k[r] = w_old * a[r] + w_new * b[r];
}

// Traces the point x (a node, or the end of an earlier trace) back over dt
// with n_sub RK4 substeps; writes X.
void departure_point(const Mesh& me, const Velocity& V, int n_sub, const double* x, double* X) {
  const int d = me.d;
  const double h = V.dt / n_sub;
  double y[3], k1[3], k2[3], k3[3], k4[3], z[3];
  for (int r = 0; r < d; ++r) y[r] = x[r];
  for (int j = 0; j < n_sub; ++j) {
    const double back = j * h;
    for (int r = 0; r < d; ++r) z[r] = y[r];
    velocity_at(me, V, back, z, k1);
    for (int r = 0; r < d; ++r) z[r] = y[r] - 0.5 * h * k1[r];
    clamp_to_box(me, z);
    velocity_at(me, V, back + 0.5 * h, z, k2);
    for (int r = 0; r < d; ++r) z[r] = y[r] - 0.5 * h * k2[r];
    clamp_to_box(me, z);
    velocity_at(me, V, back + 0.5 * h, z, k3);
    for (int r = 0; r < d; ++r) z[r] = y[r] - h * k3[r];
    clamp_to_box(me, z);
    velocity_at(me, V, back + h, z, k4);
    for (int r = 0; r < d; ++r) y[r] = y[r] - h / 6.0 * (k1[r] + 2.0 * k2[r] + 2.0 * k3[r] + k4[r]);
    clamp_to_box(me, y);
  }
  for (int r = 0; r < d; ++r) X[r] = y[r];
}

template <class F>
void parallel_for(int64_t begin, int64_t end, int nthreads, F&& f) {
  if (nthreads <= 1 || end - begin < 2) {
    for (int64_t i = begin; i < end; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  const int64_t n = end - begin;
  for (int t = 0; t < nthreads; ++t) {
    int64_t a = begin + n * t / nthreads, b = begin + n * (t + 1) / nthreads;
    pool.emplace_back([a, b, &f]() { for (int64_t i = a; i < b; ++i) f(i); });
  }
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------
// P1 / P2 mass matrix (Sec. 3.1 metrics), exact via barycentric monomial integrals:
// int_T lam_0^a0 ... lam_d^ad = d! |T| a0! ... ad! / (d + sum a)!.
// ---------------------------------------------------------------------------

struct Poly {  // polynomial in the d+1 barycentric coordinates
  std::map<std::array<int, 4>, double> c;
};

Poly basis_poly(int d, int order, int i) {
  Poly P;
  if (order == 1) {  // P1 vertex: lam_i
    std::array<int, 4> e1{0, 0, 0, 0};
    e1[i] = 1;
    P.c[e1] += 1.0;
  } else if (i <= d) {  // P2 vertex: 2 lam_i^2 - lam_i
    std::array<int, 4> e2{0, 0, 0, 0}, e1{0, 0, 0, 0};
    e2[i] = 2;
    e1[i] = 1;
    P.c[e2] += 2.0;
    P.c[e1] += -1.0;
  } else {       // edge (a, b) in the order of p2_stencil
    int n = d + 1;
    for (int a = 0; a <= d; ++a)
      for (int b = a + 1; b <= d; ++b) {
        if (n++ == i) {
          std::array<int, 4> e{0, 0, 0, 0};
          e[a] = 1;
          e[b] = 1;
          P.c[e] += 4.0;
        }
      }
  }
  return P;
}

double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

int n_basis(int d, int order) { return order == 1 ? d + 1 : (d + 1) * (d + 2) / 2; }

// Mass matrix of the reference simplex scaled to unit volume |T| = 1.
void mass_unit(int d, int order, double* Mref) {
  const int nb = n_basis(d, order);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      Poly A = basis_poly(d, order, i), B = basis_poly(d, order, j);
      double s = 0.0;
      for (auto& ta : A.c)
        for (auto& tb : B.c) {
          int tot = 0;
          double num = factorial(d);
          for (int k = 0; k <= d; ++k) {
            int e = ta.first[k] + tb.first[k];
            tot += e;
            num *= factorial(e);
          }
          s += ta.second * tb.second * num / factorial(d + tot);
        }
      Mref[i * nb + j] = s;
    }
}

// Calls f(macro, vertices w[0..d]) for every micro simplex of every macro: the
// Kuhn simplices (one per permutation) of each cell that lie in the reference
// simplex.
template <class F>
void for_each_micro_simplex(const Mesh& me, F&& f) {
  const int d = me.d, N = me.N;
  int perm[3] = {0, 1, 2};
  for (int64_t m = 0; m < (int64_t)me.mac.size(); ++m) {
    int c[3] = {0, 0, 0};
    auto cell = [&]() {
      int pm[3] = {0, 1, 2};
      do {
        int w[4][3];
        for (int r = 0; r < d; ++r) w[0][r] = c[r];
        bool inside = true;
        for (int j = 1; j <= d; ++j) {
          for (int r = 0; r < d; ++r) w[j][r] = w[j - 1][r];
          w[j][pm[j - 1]] += 1;
        }
        for (int j = 0; j <= d && inside; ++j) {
          if (w[j][0] > N) inside = false;
          for (int r = 1; r < d; ++r) if (w[j][r] > w[j][r - 1]) inside = false;
          if (w[j][d - 1] < 0) inside = false;
        }
        if (inside) f(m, w);
      } while (std::next_permutation(pm, pm + d));
    };
    (void)perm;
    if (d == 2) {
      for (c[0] = 0; c[0] < N; ++c[0])
        for (c[1] = 0; c[1] <= c[0]; ++c[1]) cell();
    } else {
      for (c[0] = 0; c[0] < N; ++c[0])
        for (c[1] = 0; c[1] <= c[0]; ++c[1])
          for (c[2] = 0; c[2] <= c[1]; ++c[2]) cell();
    }
  }
}

double simplex_volume(int d, const double V[4][3]) {
  double A[9];
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) A[r * d + c] = V[c + 1][r] - V[0][r];
  double det = (d == 2) ? A[0] * A[3] - A[1] * A[2]
                        : A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                              A[2] * (A[3] * A[7] - A[4] * A[6]);
  return std::fabs(det) / (d == 2 ? 2.0 : 6.0);
}

// ---------------------------------------------------------------------------
// Diffusion step (Eq. finite-dimensional Galerkin approximation, Eq. linear
// system): mass and stiffness matrices of every micro simplex, assembled into
// sparse M and A by the Python wrapper.  With grad phi_i = sum_k
// (dphi_i / dlam_k) grad lam_k the stiffness entry is
//   A_ij = sum_{k,l} (grad lam_k . grad lam_l) int_T (dphi_i/dlam_k)(dphi_j/dlam_l),
// every integral exact by the barycentric monomial formula above.
// ---------------------------------------------------------------------------

Poly diff_poly(const Poly& P, int k) {
  Poly D;
  for (auto& t : P.c) {
    if (t.first[k] == 0) continue;
    std::array<int, 4> e = t.first;
    const double f = t.second * e[k];
    e[k] -= 1;
    D.c[e] += f;
  }
  return D;
}

// int_T A B over a simplex of unit volume.
double integrate_unit(int d, const Poly& A, const Poly& B) {
  double s = 0.0;
  for (auto& ta : A.c)
    for (auto& tb : B.c) {
      int tot = 0;
      double num = factorial(d);
      for (int k = 0; k <= d; ++k) {
        const int e = ta.first[k] + tb.first[k];
        tot += e;
        num *= factorial(e);
      }
      s += ta.second * tb.second * num / factorial(d + tot);
    }
  return s;
}

// Gradients of the barycentric coordinates of the simplex V: for k >= 1 row
// k-1 of J^{-1}, J = [V1 - V0 | ... | Vd - V0]; grad lam_0 = -sum of the others.
void grad_lambdas(int d, const double V[4][3], double G[4][3]) {
  double J[9], I[9];
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) J[r * d + c] = V[c + 1][r] - V[0][r];
  for (int c = 0; c < d; ++c) {  // column c of J^{-1}: solve J z = e_c
    double e[3] = {0.0, 0.0, 0.0}, z[3];
    e[c] = 1.0;
    solve_small(d, J, e, z);
    for (int r = 0; r < d; ++r) I[r * d + c] = z[r];
  }
  for (int r = 0; r < 3; ++r) G[0][r] = 0.0;
  for (int k = 1; k <= d; ++k)
    for (int r = 0; r < d; ++r) {
      G[k][r] = I[(k - 1) * d + r];
      G[0][r] -= G[k][r];
    }
}

double poly_eval(const Poly& P, const double* mu) {
  double s = 0.0;
  for (auto& t : P.c) {
    double v = t.second;
    for (int k = 0; k < 4; ++k)
      for (int e = 0; e < t.first[k]; ++e) v *= mu[k];
    s += v;
  }
  return s;
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the Legendre
// recurrence).
void gauss_legendre01(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Metric of the blended stiffness at a computational point x (2D annulus,
// Sec. 2.1): G = DPhi^{-1} DPhi^{-T} |det DPhi|, so that
// int grad_y a . grad_y b dy = int grad_x a^T G grad_x b dx.  DPhi from the
// sector coordinates (lam, rho): x = rho p(lam), y = rho e(theta_k + lam Delta),
// DPhi = (dy/d(lam, rho)) (dx/d(lam, rho))^{-1}.
void blend_metric(const Blend& b, const double* x, double G[2][2]) {
  const double pi = 3.14159265358979323846;
  const double delta = 2.0 * pi / b.nsec;
  int k;
  double lam0;
  blend_sector(b, std::atan2(x[1], x[0]), &k, &lam0);
  const double tk = b.theta0 + k * delta;
  const double ek[2] = {std::cos(tk), std::sin(tk)}, ek1[2] = {std::cos(tk + delta), std::sin(tk + delta)};
  const double ck = ek[0] * x[1] - ek[1] * x[0], ck1 = ek1[0] * x[1] - ek1[1] * x[0];
  const double lam = ck / (ck - ck1);
  const double p[2] = {(1 - lam) * ek[0] + lam * ek1[0], (1 - lam) * ek[1] + lam * ek1[1]};
  const double rho = std::sqrt(x[0] * x[0] + x[1] * x[1]) / std::sqrt(p[0] * p[0] + p[1] * p[1]);
  const double th = tk + lam * delta;
  const double Jx[2][2] = {{rho * (ek1[0] - ek[0]), p[0]}, {rho * (ek1[1] - ek[1]), p[1]}};
  const double Jy[2][2] = {{-rho * delta * std::sin(th), std::cos(th)}, {rho * delta * std::cos(th), std::sin(th)}};
  const double dx = Jx[0][0] * Jx[1][1] - Jx[0][1] * Jx[1][0];
  const double Jxi[2][2] = {{Jx[1][1] / dx, -Jx[0][1] / dx}, {-Jx[1][0] / dx, Jx[0][0] / dx}};
  double D[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) D[r][c] = Jy[r][0] * Jxi[0][c] + Jy[r][1] * Jxi[1][c];
  const double det = D[0][0] * D[1][1] - D[0][1] * D[1][0];
  const double Di[2][2] = {{D[1][1] / det, -D[0][1] / det}, {-D[1][0] / det, D[0][0] / det}};
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) G[r][c] = (Di[r][0] * Di[c][0] + Di[r][1] * Di[c][1]) * std::fabs(det);
}

// Per-micro-simplex local node ids [n_simplices, nb] and matrices
// [n_simplices, nb, nb] of the mass and the stiffness; returns the number of
// micro simplices (the outputs may be null to query it).
int64_t element_matrices(const Mesh& me, int32_t* node_out, double* M_out, double* A_out) {
  const int d = me.d, nb = n_basis(d, me.order);
  std::vector<double> Mref(nb * nb);
  mass_unit(d, me.order, Mref.data());
  // Iref[((i * nb + j) * (d+1) + k) * (d+1) + l] = int_unit (dphi_i/dlam_k)(dphi_j/dlam_l)
  std::vector<double> Iref(nb * nb * (d + 1) * (d + 1));
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j)
      for (int k = 0; k <= d; ++k)
        for (int l = 0; l <= d; ++l)
          Iref[((i * nb + j) * (d + 1) + k) * (d + 1) + l] =
              integrate_unit(d, diff_poly(basis_poly(d, me.order, i), k), diff_poly(basis_poly(d, me.order, j), l));
  int64_t n = 0;
  for_each_micro_simplex(me, [&](int64_t m, int w[4][3]) {
    if (node_out) {
      Located lc;
      lc.macro = m;
      for (int j = 0; j <= d; ++j)
        for (int r = 0; r < d; ++r) lc.w[j][r] = w[j][r];
      for (int j = 0; j < 4; ++j) lc.mu[j] = 0.0;
      double phi[10];
      stencil(me, lc, node_out + n * nb, phi);
      double V[4][3], G[4][3];
      for (int j = 0; j <= d; ++j) {
        int wt[4];
        lattice_weights(d, me.N, w[j], wt);
        lattice_point(me.mac[m], d, wt, me.N, V[j]);
      }
      const double vol = simplex_volume(d, V);
      grad_lambdas(d, V, G);
      double* Me = M_out + n * nb * nb;
      double* Ae = A_out + n * nb * nb;
      if (me.bl.on) {
        // blended (2D): det DPhi = Delta / sin(Delta) scales the mass; the
        // stiffness by a 5 x 5 collapsed Gauss rule with the metric above
        const double delta = 2.0 * 3.14159265358979323846 / me.bl.nsec;
        const double jac = delta / std::sin(delta);
        for (int i = 0; i < nb * nb; ++i) {
          Me[i] = vol * Mref[i] * jac;
          Ae[i] = 0.0;
        }
        double gx[5], gw[5];
        gauss_legendre01(5, gx, gw);
        for (int a = 0; a < 5; ++a)
          for (int bq = 0; bq < 5; ++bq) {
            const double u = gx[a], v = gx[bq];
            const double mu[4] = {1.0 - u - v * (1.0 - u), u, v * (1.0 - u), 0.0};
            const double W = gw[a] * gw[bq] * (1.0 - u) * 2.0 * vol;
            double xq[2] = {0.0, 0.0};
            for (int j = 0; j <= 2; ++j)
              for (int r = 0; r < 2; ++r) xq[r] += mu[j] * V[j][r];
            double Gm[2][2];
            blend_metric(me.bl, xq, Gm);
            double gr[10][2];
            for (int i = 0; i < nb; ++i) {
              gr[i][0] = gr[i][1] = 0.0;
              for (int k = 0; k <= 2; ++k) {
                const double dk = poly_eval(diff_poly(basis_poly(2, me.order, i), k), mu);
                gr[i][0] += dk * G[k][0];
                gr[i][1] += dk * G[k][1];
              }
            }
            for (int i = 0; i < nb; ++i)
              for (int j = 0; j < nb; ++j)
                Ae[i * nb + j] += W * (gr[i][0] * (Gm[0][0] * gr[j][0] + Gm[0][1] * gr[j][1]) +
                                       gr[i][1] * (Gm[1][0] * gr[j][0] + Gm[1][1] * gr[j][1]));
          }
        ++n;
        return;
      }
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
          Me[i * nb + j] = vol * Mref[i * nb + j];
          double a = 0.0;
          for (int k = 0; k <= d; ++k)
            for (int l = 0; l <= d; ++l) {
              double g = 0.0;
              for (int r = 0; r < d; ++r) g += G[k][r] * G[l][r];
              a += g * Iref[((i * nb + j) * (d + 1) + k) * (d + 1) + l];
            }
          Ae[i * nb + j] = vol * a;
        }
    }
    ++n;
  });
  return n;
}

// Nodes on the boundary of the macro mesh: a node lies on face k of a macro
// where its barycentric weight k is 0; the face is a boundary face when no
// other macro shares its vertices.
void boundary_nodes(const Mesh& me, uint8_t* out) {
  const int d = me.d;
  std::map<std::array<int64_t, 3>, int> count;
  auto face_key = [&](const Macro& mc, int k) {
    std::array<int64_t, 3> f{-1, -1, -1};
    int n = 0;
    for (int j = 0; j <= d; ++j)
      if (j != k) f[n++] = mc.v[j];
    std::sort(f.begin(), f.begin() + d);
    return f;
  };
  for (auto& mc : me.mac)
    for (int k = 0; k <= d; ++k) count[face_key(mc, k)] += 1;
  std::fill(out, out + me.n_nodes, uint8_t(0));
  for (int64_t m = 0; m < (int64_t)me.mac.size(); ++m) {
    bool bface[4] = {false, false, false, false};
    for (int k = 0; k <= d; ++k) bface[k] = count[face_key(me.mac[m], k)] == 1;
    for_each_lattice_point(d, me.M, [&](const int* p) {
      int w[4];
      lattice_weights(d, me.M, p, w);
      for (int k = 0; k <= d; ++k)
        if (w[k] == 0 && bface[k]) out[me.id[m][me.dense(p)]] = 1;
    });
  }
}

// ---------------------------------------------------------------------------
// Forward-mode directional derivatives (dual numbers) of the advection step
// with respect to the nodal velocity: each velocity value u_j becomes
// u_j + eps v_j and every operation of the step above is repeated on pairs
// (value, derivative).  Discrete decisions (macro choice, micro element,
// pivots, clamps) are taken on the values; a clamped coordinate has zero
// derivative.  Used only to check the adjoint kernel.
// ---------------------------------------------------------------------------

struct Dual {
  double v = 0.0, d = 0.0;
};
Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }

// Barycentric coordinates of a dual point with respect to a fixed simplex.
void barycentric_dual(int d, const double V[4][3], const Dual* y, Dual* lam) {
  Dual A[4][5];
  const int n = d + 1;
  for (int r = 0; r < d; ++r) {
    for (int c = 0; c < n; ++c) A[r][c] = {V[c][r], 0.0};
    A[r][n] = y[r];
  }
  for (int c = 0; c < n; ++c) A[d][c] = {1.0, 0.0};
  A[d][n] = {1.0, 0.0};
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r][col].v) > std::fabs(A[piv][col].v)) piv = r;
    if (piv != col)
      for (int j = 0; j <= n; ++j) std::swap(A[piv][j], A[col][j]);
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      Dual f = A[r][col] / A[col][col];
      for (int j = col; j <= n; ++j) A[r][j] = A[r][j] - f * A[col][j];
    }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i][n] / A[i][i];
}

void clamp_to_box_dual(const Mesh& me, Dual* y) {
  for (int r = 0; r < me.d; ++r) {
    if (y[r].v < me.lo[r]) y[r] = {me.lo[r], 0.0};
    if (y[r].v > me.hi[r]) y[r] = {me.hi[r], 0.0};
  }
}

// Field evaluation with dual point and dual nodal values (F + eps dF).
void eval_field_dual(const Mesh& me, const double* F, const double* dF, int ncomp, Dual* y, Dual* out) {
  const int d = me.d;
  double yv[3];
  for (int r = 0; r < d; ++r) yv[r] = y[r].v;
  Located lc;
  locate(me, yv, lc);  // decisions on the values (may move yv onto the mesh)
  for (int r = 0; r < d; ++r)
    if (yv[r] != y[r].v) y[r] = {yv[r], 0.0};
  double V[4][3];
  for (int j = 0; j <= d; ++j) {
    int wt[4];
    lattice_weights(d, me.N, lc.w[j], wt);
    lattice_point(me.mac[lc.macro], d, wt, me.N, V[j]);
  }
  Dual mu[4];
  barycentric_dual(d, V, y, mu);
  int32_t node[10];
  double phi_unused[10];
  const int n = stencil(me, lc, node, phi_unused);
  Dual phi[10];
  int k = 0;
  if (me.order == 1) {
    for (int v = 0; v <= d; ++v) phi[k++] = mu[v];
  } else {
    for (int v = 0; v <= d; ++v) phi[k++] = mu[v] * (2.0 * mu[v] - Dual{1.0, 0.0});
    for (int a = 0; a <= d; ++a)
      for (int b = a + 1; b <= d; ++b) phi[k++] = 4.0 * (mu[a] * mu[b]);
  }
  for (int c = 0; c < ncomp; ++c) {
    Dual s{0.0, 0.0};
    for (int j = 0; j < n; ++j) {
      const int64_t id = int64_t(node[j]) * ncomp + c;
      s = s + phi[j] * Dual{F[id], dF ? dF[id] : 0.0};
    }
    out[c] = s;
  }
}

struct VelocityDual {
  const double* u_old;
  const double* u_new;
  const double* du_old;
  const double* du_new;
  double dt;
};

void velocity_at_dual(const Mesh& me, const VelocityDual& V, double back, Dual* y, Dual* k) {
  const int d = me.d;
  Dual a[3], b[3];
  eval_field_dual(me, V.u_new, V.du_new, d, y, b);
  if (V.u_old == V.u_new) {
    for (int r = 0; r < d; ++r) k[r] = b[r];
    return;
  }
  eval_field_dual(me, V.u_old, V.du_old, d, y, a);
  const double w_old = back / V.dt, w_new = (V.dt - back) / V.dt;
  for (int r = 0; r < d; ++r) k[r] = w_old * a[r] + w_new * b[r];
}

void departure_point_dual(const Mesh& me, const VelocityDual& V, int n_sub, const double* x, Dual* X) {
  const int d = me.d;
  const double h = V.dt / n_sub;
  Dual y[3], k1[3], k2[3], k3[3], k4[3], z[3];
  for (int r = 0; r < d; ++r) y[r] = {x[r], 0.0};
  for (int j = 0; j < n_sub; ++j) {
    const double back = j * h;
    for (int r = 0; r < d; ++r) z[r] = y[r];
    velocity_at_dual(me, V, back, z, k1);
    for (int r = 0; r < d; ++r) z[r] = y[r] - (0.5 * h) * k1[r];
    clamp_to_box_dual(me, z);
    velocity_at_dual(me, V, back + 0.5 * h, z, k2);
    for (int r = 0; r < d; ++r) z[r] = y[r] - (0.5 * h) * k2[r];
    clamp_to_box_dual(me, z);
    velocity_at_dual(me, V, back + 0.5 * h, z, k3);
    for (int r = 0; r < d; ++r) z[r] = y[r] - h * k3[r];
    clamp_to_box_dual(me, z);
    velocity_at_dual(me, V, back + h, z, k4);
    for (int r = 0; r < d; ++r) y[r] = y[r] - (h / 6.0) * (k1[r] + 2.0 * k2[r] + 2.0 * k3[r] + k4[r]);
    clamp_to_box_dual(me, y);
  }
  for (int r = 0; r < d; ++r) X[r] = y[r];
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the Python wrapper in oracle/__init__.py.
// ---------------------------------------------------------------------------
extern "C" {

void* orc_mesh_create(int dim, int64_t nv, const double* xyz, int64_t nm, const int64_t* mv, int level, int order) {
  return build_mesh(dim, nv, xyz, nm, mv, level, order);
}

void orc_mesh_destroy(void* h) { delete static_cast<Mesh*>(h); }

int64_t orc_num_nodes(void* h) { return static_cast<Mesh*>(h)->n_nodes; }

void orc_node_coords(void* h, double* out) {
  Mesh* me = static_cast<Mesh*>(h);
  std::memcpy(out, me->X.data(), me->X.size() * sizeof(double));
}

// Lattice coordinates p (M >= p1 >= ... >= pd >= 0) of the macro's nodes, in
// the order (p1, p2, p3) lexicographic, with the global node number of each.
int64_t orc_macro_nodes(void* h, int64_t macro, int32_t* p_out, int32_t* node_out) {
  Mesh* me = static_cast<Mesh*>(h);
  int64_t n = 0;
  for_each_lattice_point(me->d, me->M, [&](const int* p) {
    if (p_out) for (int r = 0; r < me->d; ++r) p_out[n * me->d + r] = p[r];
    if (node_out) node_out[n] = me->id[macro][me->dense(p)];
    ++n;
  });
  return n;
}

// Locates points (after the box clamp): macro id, micro vertices (q-lattice
// points, [npts, d+1, d]) and the micro barycentric coordinates.
void orc_locate(void* h, int64_t npts, const double* pts, int64_t* macro, int32_t* wv, double* mu) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  for (int64_t i = 0; i < npts; ++i) {
    double y[3];
    for (int r = 0; r < d; ++r) y[r] = pts[i * d + r];
    clamp_to_box(*me, y);
    Located lc;
    locate(*me, y, lc);
    macro[i] = lc.macro;
    for (int j = 0; j <= d; ++j)
      for (int r = 0; r < d; ++r) wv[(i * (d + 1) + j) * d + r] = lc.w[j][r];
    for (int j = 0; j <= d; ++j) mu[i * (d + 1) + j] = lc.mu[j];
  }
}

// P1 / P2 interpolation of a field ([n_nodes, ncomp]) at arbitrary points.
void orc_eval(void* h, const double* F, int ncomp, int64_t npts, const double* pts, double* out, int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  parallel_for(0, npts, nthreads, [&](int64_t i) {
    double y[3];
    for (int r = 0; r < d; ++r) y[r] = pts[i * d + r];
    clamp_to_box(*me, y);
    eval_field(*me, F, ncomp, y, out + i * ncomp);
  });
}

// Departure points X_i of nodes [begin, end) ([n, d] output rows begin..end-1).
void orc_departure(void* h, const double* u_old, const double* u_new, double dt, int n_sub,
                   int64_t begin, int64_t end, double* X, int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  Velocity V{u_old, u_new, dt};
  parallel_for(begin, end, nthreads, [&](int64_t i) {
    departure_point(*me, V, n_sub, &me->X[i * d], X + (i - begin) * d);
  });
}

// Continues backward traces (Sec. 2.3.3): each point X_in[k] is traced back
// over dt with the velocity pair (u_old at the start of the interval, u_new
// at its end) and n_sub RK4 substeps; X_out[k] receives the new point.
void orc_trace(void* h, const double* u_old, const double* u_new, double dt, int n_sub, int64_t npts,
               const double* X_in, double* X_out, int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  Velocity V{u_old, u_new, dt};
  parallel_for(0, npts, nthreads, [&](int64_t i) {
    double x[3];
    for (int r = 0; r < d; ++r) x[r] = X_in[i * d + r];
    clamp_to_box(*me, x);
    departure_point(*me, V, n_sub, x, X_out + i * d);
  });
}

// One advection step for nodes [begin, end): T_new[i] = T^n_h(X_i) (step (iii)).
void orc_advect(void* h, const double* u_old, const double* u_new, const double* T_old, double* T_new,
                double dt, int n_sub, int64_t begin, int64_t end, int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  Velocity V{u_old, u_new, dt};
  parallel_for(begin, end, nthreads, [&](int64_t i) {
    double X[3];
    departure_point(*me, V, n_sub, &me->X[i * d], X);
    double v;
    eval_field(*me, T_old, 1, X, &v);
    T_new[i - begin] = v;
  });
}

// One advection step for the listed nodes only: out[k] = T^n_h(X_{idx[k]}).
void orc_advect_nodes(void* h, const double* u_old, const double* u_new, const double* T_old, double dt,
                      int n_sub, int64_t n_idx, const int64_t* idx, double* out, int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  Velocity V{u_old, u_new, dt};
  parallel_for(0, n_idx, nthreads, [&](int64_t k) {
    double X[3];
    departure_point(*me, V, n_sub, &me->X[idx[k] * d], X);
    eval_field(*me, T_old, 1, X, out + k);
  });
}

// Directional derivative of one advection step with respect to the nodal
// velocity in the direction (du_old, du_new): out[i] = T_new[i],
// jvp[i] = d/deps T_new[i](u + eps du), nodes [begin, end).
void orc_advect_jvp(void* h, const double* u_old, const double* u_new, const double* du_old, const double* du_new,
                    const double* T_old, double dt, int n_sub, int64_t begin, int64_t end, double* out, double* jvp,
                    int nthreads) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  VelocityDual V{u_old, u_new, du_old, du_new, dt};
  parallel_for(begin, end, nthreads, [&](int64_t i) {
    Dual X[3];
    departure_point_dual(*me, V, n_sub, &me->X[i * d], X);
    Dual v;
    eval_field_dual(*me, T_old, nullptr, 1, X, &v);
    out[i - begin] = v.v;
    jvp[i - begin] = v.d;
  });
}

// Transpose of the interpolation: g_old[j] += sum_i phi_j(X_i) g_new[i].
void orc_advect_transpose(void* h, const double* u_old, const double* u_new, const double* g_new,
                          double* g_old, double dt, int n_sub) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  Velocity V{u_old, u_new, dt};
  std::fill(g_old, g_old + me->n_nodes, 0.0);
  for (int64_t i = 0; i < me->n_nodes; ++i) {
    double X[3];
    departure_point(*me, V, n_sub, &me->X[i * d], X);
    Located lc;
    locate(*me, X, lc);
    int32_t node[10];
    double phi[10];
    int n = stencil(*me, lc, node, phi);
    for (int j = 0; j < n; ++j) g_old[node[j]] += phi[j] * g_new[i];
  }
}

// Mass-matrix products for the metrics of Sec. 3.1: out[k] = a_k^T M b_k for
// the nvec column pairs (a, b given node-major [n_nodes, nvec]).
void orc_mass_products(void* h, int nvec, const double* a, const double* b, double* out) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;

  const int nb = n_basis(d, me->order);
  std::vector<double> Mref(nb * nb);
  mass_unit(d, me->order, Mref.data());
  for (int k = 0; k < nvec; ++k) out[k] = 0.0;
  for_each_micro_simplex(*me, [&](int64_t m, int w[4][3]) {
    Located lc;
    lc.macro = m;
    for (int j = 0; j <= d; ++j)
      for (int r = 0; r < d; ++r) lc.w[j][r] = w[j][r];
    for (int j = 0; j < 4; ++j) lc.mu[j] = 0.0;
    int32_t node[10];
    double phi[10];
    stencil(*me, lc, node, phi);
    double V[4][3];
    for (int j = 0; j <= d; ++j) {
      int wt[4];
      lattice_weights(d, me->N, w[j], wt);
      lattice_point(me->mac[m], d, wt, me->N, V[j]);
    }
    const double vol = simplex_volume(d, V);
    for (int k = 0; k < nvec; ++k) {
      double s = 0.0;
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j)
          s += a[int64_t(node[i]) * nvec + k] * Mref[i * nb + j] * b[int64_t(node[j]) * nvec + k];
      out[k] += vol * s;
    }
  });
  // blended annulus: det DPhi = Delta / sin(Delta) on the whole mesh
  if (me->bl.on) {
    const double delta = 2.0 * 3.14159265358979323846 / me->bl.nsec;
    for (int k = 0; k < nvec; ++k) out[k] *= delta / std::sin(delta);
  }
}

// Every micro simplex: macro id and vertex lattice points ([count, d+1, d]).
int64_t orc_micro_simplices(void* h, int64_t* macro, int32_t* wv) {
  Mesh* me = static_cast<Mesh*>(h);
  const int d = me->d;
  int64_t n = 0;
  for_each_micro_simplex(*me, [&](int64_t m, int w[4][3]) {
    if (macro) macro[n] = m;
    if (wv)
      for (int j = 0; j <= d; ++j)
        for (int r = 0; r < d; ++r) wv[(n * (d + 1) + j) * d + r] = w[j][r];
    ++n;
  });
  return n;
}

// Local node ids, mass and stiffness matrices of every micro simplex (see
// element_matrices); returns the number of micro simplices.
int64_t orc_element_matrices(void* h, int32_t* node_out, double* M_out, double* A_out) {
  return element_matrices(*static_cast<Mesh*>(h), node_out, M_out, A_out);
}

// 1 for nodes on the boundary of the mesh, else 0 ([n_nodes]).
void orc_boundary_nodes(void* h, uint8_t* out) { boundary_nodes(*static_cast<Mesh*>(h), out); }

// Turns a 2D ring mesh into a blended annulus (see Blend): node coordinates
// become physical.  Returns 0 on success, -1 if the mesh is not such a ring.
int orc_set_annulus(void* h, double rmin, double rmax, int nsec, double theta0) {
  Mesh* me = static_cast<Mesh*>(h);
  if (me->d != 2 || nsec < 3 || !(rmin > 0.0) || !(rmax > rmin)) return -1;
  me->bl.on = true;
  me->bl.rmin = rmin;
  me->bl.rmax = rmax;
  me->bl.nsec = nsec;
  me->bl.theta0 = theta0;
  for (int64_t i = 0; i < me->n_nodes; ++i) {
    double xc[2] = {me->X[i * 2], me->X[i * 2 + 1]};
    blend_phi(me->bl, xc, &me->X[i * 2]);
  }
  return 0;
}

// Reference P1 / P2 mass matrix for a simplex of unit volume ([nb, nb]).
void orc_mass_unit(int d, int order, double* out) { mass_unit(d, order, out); }

}  // extern "C"
