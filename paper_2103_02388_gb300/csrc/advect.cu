// advect.cu -- the MMOC advection step on sm_103a (arXiv 2103.02388, Sec. 3
// steps (i)-(iii), Eq. departure point, Eq. linear interpolation,
// Algorithm 1 lines 3-4).
//
// One thread per storage node.  A thread creates its particle at node x_i
// (step (i)), traces it backwards with n_sub classic RK4 substeps through the
// P2 velocity (step (ii)) and interpolates T^n at the departure point
// (step (iii)).  All macros are resident in HBM, so the paper's particle
// migration between processes becomes an in-register macro walk.  A node on
// a macro interface is stored once per macro holding it; the thread of every
// copy traces the owner copy (same macro frame, same instructions), so all
// copies receive bitwise the same value and no synchronisation pass is needed
// (the single-owner rule of Sec. 3 "Grid data structure").
//
// Point representation.  A point is kept as an offset d from its start node
// x_i, and its level-L lattice coordinate in the current macro m as
// q = b + r0 + NJinv_m d with an integer part b and a small fraction r0 of
// the start node.  The integer part carries the node's absolute position
// exactly, so FP32 keeps full precision in the fractional coordinates that
// decide the micro element, independent of the macro's size.
//
// Field evaluation (Sec. 3 "Field evaluation"):
//   macro   -- barycentrics l = (N - q1, q1 - q2, q2 - q3, q3) in lattice
//              units; if min l < -tol the walk hops across the face opposite
//              the most negative one (at most kMaxHops hops);
//   micro   -- cell c = floor(q), fractions f = q - c; the Kuhn simplex of
//              the cell is given by the descending order of f (O(1));
//   P2 sum  -- micro barycentrics L = (1 - f_s0, f_s0 - f_s1, f_s1 - f_s2,
//              f_s2); vertex basis L(2L - 1), edge basis 4 L_a L_b.
// In FP32, a macro decision whose barycentric lies within kBand32 of 0 is
// re-taken in FP64 from the exact start node.
#include <cstdint>

#include "elm_internal.h"

namespace elm {
namespace {

constexpr double kTol64 = 1e-9;     // "inside" tolerance, lattice units (FP64)
constexpr float kBand32 = 3e-5f;    // FP32 tie band re-decided in FP64, lattice units

template <class R>
struct Tables;

template <>
struct Tables<double> {
  const MacroGeo* g;
  __device__ double nj(int m, int k) const { return g[m].NJinv[k]; }
  __device__ double J(int m, int k) const { return g[m].J[k]; }
  __device__ double v0(int m, int k) const { return g[m].v0[k]; }
  __device__ int nb(int m, int k) const { return g[m].nb[k]; }
};

template <>
struct Tables<float> {
  const MacroGeo32* g;
  __device__ float nj(int m, int k) const { return g[m].NJinv[k]; }
  __device__ float J(int m, int k) const { return g[m].J[k]; }
  __device__ float v0(int m, int k) const { return g[m].v0[k]; }
  __device__ int nb(int m, int k) const { return g[m].nb[k]; }
};

__device__ __forceinline__ int tri2(int k) { return k * (k + 1) / 2; }
__device__ __forceinline__ int tri3(int k) { return k * (k + 1) * (k + 2) / 6; }

// Storage slot within a macro -> lattice point p (packed order p1, p2[, p3]).
template <int D>
__device__ __forceinline__ void unpack(int r, int* p) {
  if (D == 3) {
    int p1 = __float2int_rd(cbrtf(6.0f * float(r)));
    while (p1 > 0 && tri3(p1) > r) --p1;
    while (tri3(p1 + 1) <= r) ++p1;
    r -= tri3(p1);
    int p2 = __float2int_rd((sqrtf(8.0f * float(r) + 1.0f) - 1.0f) * 0.5f);
    while (p2 > 0 && tri2(p2) > r) --p2;
    while (tri2(p2 + 1) <= r) ++p2;
    p[0] = p1;
    p[1] = p2;
    p[2] = r - tri2(p2);
  } else {
    int p1 = __float2int_rd((sqrtf(8.0f * float(r) + 1.0f) - 1.0f) * 0.5f);
    while (p1 > 0 && tri2(p1) > r) --p1;
    while (tri2(p1 + 1) <= r) ++p1;
    p[0] = p1;
    p[1] = r - tri2(p1);
  }
}

template <int D>
__device__ __forceinline__ int packed(const int* p) {
  return D == 3 ? tri3(p[0]) + tri2(p[1]) + p[2] : tri2(p[0]) + p[1];
}

// Per-thread tracing state.
template <int D, class R>
struct Tracer {
  // launch constants (copied, so no kernel parameter is addressed)
  const MacroGeo* geo;   // FP64 macro table (start-node frames, tie-breaks)
  Tables<R> tab;         // macro table in the working precision
  int N;
  int64_t npm;
  const R* un;
  const R* uo;
  const R* T;
  int steady;
  R dt;
  unsigned* status;
  int m0;          // home macro
  int p[D];        // home lattice point
  // current frame: q = b + r0 + nj * d
  int m;
  int b[D];
  R r0[D];
  R nj[D * D];
  R dlo[D], dhi[D];  // box limits as offsets from x_i

  __device__ void load_nj(int mm) {
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) nj[r * D + c] = tab.nj(mm, r * 3 + c);
  }

  __device__ void home_frame() {
    m = m0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      b[k] = p[k] >> 1;
      r0[k] = (p[k] & 1) ? R(0.5) : R(0);
    }
    load_nj(m0);
  }

  // Exact (FP64) start node position.
  __device__ void node_position64(double* x) const {
    const MacroGeo& g = geo[m0];
    const double invM = 1.0 / double(2 * N);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double s = g.v0[r];
#pragma unroll
      for (int c = 0; c < D; ++c) s = fma(g.J[r * 3 + c], double(p[c]) * invM, s);
      x[r] = s;
    }
  }

  // Lattice coordinate of the start node in macro mm, FP64.
  __device__ void node_lattice64(int mm, double* q) const {
    double x[D];
    node_position64(x);
    const MacroGeo& g = geo[mm];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) s = fma(g.NJinv[r * 3 + c], x[c] - g.v0[c], s);
      q[r] = s;
    }
  }

  __device__ void foreign_frame(int mm) {
    if (mm == m0) {
      home_frame();
      return;
    }
    double q[D];
    node_lattice64(mm, q);
    m = mm;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double fl = floor(q[k]);
      b[k] = int(fl);
      r0[k] = R(q[k] - fl);
    }
    load_nj(mm);
  }

  // Macro barycentrics in lattice units from the split coordinate (c, f).
  __device__ static void bary(int N, const int* c, const R* f, R* l) {
    l[0] = R(N - c[0]) - f[0];
#pragma unroll
    for (int k = 1; k < D; ++k) l[k] = R(c[k - 1] - c[k]) + (f[k - 1] - f[k]);
    l[D] = R(c[D - 1]) + f[D - 1];
  }

  // FP64 barycentrics of the point x_i + d in the current macro.
  __device__ void bary64(const R* d, double* l) const {
    double q[D];
    node_lattice64(m, q);
    const MacroGeo& g = geo[m];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) q[r] = fma(g.NJinv[r * 3 + c], double(d[c]), q[r]);
    l[0] = double(N) - q[0];
#pragma unroll
    for (int k = 1; k < D; ++k) l[k] = q[k - 1] - q[k];
    l[D] = q[D - 1];
  }

  // Locates x_i + d: walks macros from the current frame, returns the micro
  // cell c and fractions f (retracted into the macro's reference simplex).
  __device__ void locate(const R* d, int* c, R* f) {
    for (int hop = 0;; ++hop) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R r = r0[k];
#pragma unroll
        for (int j = 0; j < D; ++j) r = fma(nj[k * D + j], d[j], r);
        const R fl = floor(r);
        c[k] = b[k] + int(fl);
        f[k] = r - fl;
      }
      R l[D + 1];
      bary(N, c, f, l);
      int kmin = 0;
      R lmin = l[0];
#pragma unroll
      for (int k = 1; k <= D; ++k)
        if (l[k] < lmin) {
          lmin = l[k];
          kmin = k;
        }
      bool outside;
      if (sizeof(R) == 4) {
        outside = lmin < R(-kBand32);
        if (!outside && lmin < R(kBand32)) {
          // tie band: decide in FP64 from the exact start node
          double l64[D + 1];
          bary64(d, l64);
          double m64 = l64[0];
          int k64 = 0;
#pragma unroll
          for (int k = 1; k <= D; ++k)
            if (l64[k] < m64) {
              m64 = l64[k];
              k64 = k;
            }
          outside = m64 < -kTol64;
          kmin = k64;
        }
      } else {
        outside = lmin < R(-kTol64);
      }
      if (!outside) break;
      const int nb = tab.nb(m, kmin);
      if (nb < 0) break;  // outside the mesh: the retraction below clamps
      if (hop >= kMaxHops) {
        atomicOr(status, kFlagWalkLimit);
        break;
      }
      foreign_frame(nb);
    }
    // Retraction into N >= q1 >= q2 (>= q3) >= 0 on the split coordinate.
    if (c[0] < 0) { c[0] = 0; f[0] = R(0); }
    if (c[0] > N - 1) { c[0] = N - 1; f[0] = R(1); }
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (c[k] > c[k - 1] || (c[k] == c[k - 1] && f[k] > f[k - 1])) { c[k] = c[k - 1]; f[k] = f[k - 1]; }
      if (c[k] < 0) { c[k] = 0; f[k] = R(0); }
    }
  }

  // P2 stencil of the micro simplex holding (c, f): storage slots and basis.
  __device__ void stencil(const int* c, const R* f, int64_t* slot, R* phi) const {
    // descending order of f, ties by axis (stable)
    int s[D];
    R fs[D];
#pragma unroll
    for (int k = 0; k < D; ++k) { s[k] = k; fs[k] = f[k]; }
    auto cswap = [&](int i, int j) {
      if (fs[j] > fs[i]) {
        R t = fs[i]; fs[i] = fs[j]; fs[j] = t;
        int u = s[i]; s[i] = s[j]; s[j] = u;
      }
    };
    if (D == 3) { cswap(0, 1); cswap(1, 2); cswap(0, 1); } else { cswap(0, 1); }
    // micro vertices w_v = c + e_s0 + .. + e_s(v-1); barycentrics L
    int w[D + 1][D];
    R L[D + 1];
#pragma unroll
    for (int k = 0; k < D; ++k) w[0][k] = c[k];
#pragma unroll
    for (int v = 1; v <= D; ++v) {
#pragma unroll
      for (int k = 0; k < D; ++k) w[v][k] = w[v - 1][k] + (s[v - 1] == k ? 1 : 0);
    }
    L[0] = R(1) - fs[0];
#pragma unroll
    for (int v = 1; v < D; ++v) L[v] = fs[v - 1] - fs[v];
    L[D] = fs[D - 1];
    const int64_t base = int64_t(m) * npm;
    int n = 0;
#pragma unroll
    for (int v = 0; v <= D; ++v) {
      int q[D];
#pragma unroll
      for (int k = 0; k < D; ++k) q[k] = 2 * w[v][k];
      slot[n] = base + packed<D>(q);
      phi[n] = L[v] * (R(2) * L[v] - R(1));
      ++n;
    }
#pragma unroll
    for (int i = 0; i <= D; ++i)
#pragma unroll
      for (int j = i + 1; j <= D; ++j) {
        int q[D];
#pragma unroll
        for (int k = 0; k < D; ++k) q[k] = w[i][k] + w[j][k];
        slot[n] = base + packed<D>(q);
        phi[n] = R(4) * L[i] * L[j];
        ++n;
      }
  }

  __device__ void clamp_box(R* d) const {
#pragma unroll
    for (int k = 0; k < D; ++k) d[k] = fmin(fmax(d[k], dlo[k]), dhi[k]);
  }

  // Velocity u~ at x_i + d at backward time `back` (Eq. linear interpolation).
  __device__ void velocity(const R* d, R back, R* k) {
    constexpr int NB = (D + 1) * (D + 2) / 2;
    int c[D];
    R f[D];
    locate(d, c, f);
    int64_t slot[NB];
    R phi[NB];
    stencil(c, f, slot, phi);
#pragma unroll
    for (int r = 0; r < D; ++r) k[r] = R(0);
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int r = 0; r < D; ++r) k[r] = fma(phi[j], __ldg(un + slot[j] * D + r), k[r]);
    if (!steady) {
      R ko[D];
#pragma unroll
      for (int r = 0; r < D; ++r) ko[r] = R(0);
#pragma unroll
      for (int j = 0; j < NB; ++j)
#pragma unroll
        for (int r = 0; r < D; ++r) ko[r] = fma(phi[j], __ldg(uo + slot[j] * D + r), ko[r]);
      const R w_old = back / dt, w_new = (dt - back) / dt;
#pragma unroll
      for (int r = 0; r < D; ++r) k[r] = w_old * ko[r] + w_new * k[r];
    }
  }

  __device__ R scalar(const R* d) {
    constexpr int NB = (D + 1) * (D + 2) / 2;
    int c[D];
    R f[D];
    locate(d, c, f);
    int64_t slot[NB];
    R phi[NB];
    stencil(c, f, slot, phi);
    R v = R(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) v = fma(phi[j], __ldg(T + slot[j]), v);
    return v;
  }
};

template <int D, class R>
__global__ void __launch_bounds__(256) k_advect(AdvectArgs args, Tables<R> tab) {
  const int64_t slot = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (slot >= args.n_storage) return;
  Tracer<D, R> t;
  t.geo = args.geo;
  t.tab = tab;
  t.N = args.N;
  t.npm = args.npm;
  t.un = static_cast<const R*>(args.u_new);
  t.uo = static_cast<const R*>(args.u_old);
  t.T = static_cast<const R*>(args.T_old);
  t.steady = args.steady;
  t.dt = R(args.dt);
  t.status = args.status;
  // (i) particle creation at the node (interface copies trace their owner)
  t.m0 = int(slot / args.npm);
  unpack<D>(int(slot - int64_t(t.m0) * args.npm), t.p);
  {
    const int M = 2 * args.N;
    bool iface = t.p[0] == M || t.p[D - 1] == 0;
#pragma unroll
    for (int k = 1; k < D; ++k) iface = iface || t.p[k] == t.p[k - 1];
    if (iface) {
      const int64_t own = args.owner[args.unique_map[slot]];
      if (own != slot) {
        t.m0 = int(own / args.npm);
        unpack<D>(int(own - int64_t(t.m0) * args.npm), t.p);
      }
    }
  }
  {
    const R invM = R(1) / R(2 * args.N);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      R x = tab.v0(t.m0, r);
#pragma unroll
      for (int c = 0; c < D; ++c) x = fma(tab.J(t.m0, r * 3 + c), R(t.p[c]) * invM, x);
      t.dlo[r] = R(args.lo[r]) - x;
      t.dhi[r] = R(args.hi[r]) - x;
    }
  }
  t.home_frame();
  // (ii) backward RK4, n_sub substeps of h = dt / n_sub
  const R h = R(args.dt) / R(args.n_sub);
  const R* un = t.un;
  R d[D], k1[D], k[D], acc[D], z[D];
#pragma unroll
  for (int r = 0; r < D; ++r) d[r] = R(0);
  bool finite = true;
  for (int j = 0; j < args.n_sub; ++j) {
    const R back = R(j) * h;
    if (j == 0) {
      // the first stage sits on the node: the P2 interpolant is the nodal value
#pragma unroll
      for (int r = 0; r < D; ++r) k1[r] = __ldg(un + slot * D + r);
    } else {
      t.velocity(d, back, k1);
    }
#pragma unroll
    for (int r = 0; r < D; ++r) { acc[r] = k1[r]; z[r] = d[r] - R(0.5) * h * k1[r]; }
    t.clamp_box(z);
    t.velocity(z, back + R(0.5) * h, k);
#pragma unroll
    for (int r = 0; r < D; ++r) { acc[r] = fma(R(2), k[r], acc[r]); z[r] = d[r] - R(0.5) * h * k[r]; }
    t.clamp_box(z);
    t.velocity(z, back + R(0.5) * h, k);
#pragma unroll
    for (int r = 0; r < D; ++r) { acc[r] = fma(R(2), k[r], acc[r]); z[r] = d[r] - h * k[r]; }
    t.clamp_box(z);
    t.velocity(z, back + h, k);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      acc[r] += k[r];
      finite = finite && isfinite(acc[r]);
      d[r] = d[r] - h / R(6) * acc[r];
    }
    t.clamp_box(d);
  }
  // (iii) temperature at the departure point
  const R v = t.scalar(d);
  finite = finite && isfinite(v);
  if (!finite) atomicOr(args.status, kFlagNonFinite);
  static_cast<R*>(args.T_new)[slot] = v;
}

template <class R>
__global__ void k_gather(const R* __restrict__ in, R* __restrict__ out, const int64_t* __restrict__ idx,
                         int64_t n, int ncomp) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * ncomp) return;
  const int64_t node = i / ncomp;
  const int c = int(i - node * ncomp);
  out[i] = in[idx[node] * ncomp + c];
}

}  // namespace

cudaError_t launch_advect(int dim, int precision, const AdvectArgs& a, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = (a.n_storage + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  if (precision == ELM_FP64) {
    Tables<double> t{a.geo};
    if (dim == 3) k_advect<3, double><<<unsigned(blocks), threads, 0, s>>>(a, t);
    else k_advect<2, double><<<unsigned(blocks), threads, 0, s>>>(a, t);
  } else {
    Tables<float> t{a.geo32};
    if (dim == 3) k_advect<3, float><<<unsigned(blocks), threads, 0, s>>>(a, t);
    else k_advect<2, float><<<unsigned(blocks), threads, 0, s>>>(a, t);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(int precision, const void* in, void* out, const int64_t* idx, int64_t n, int ncomp,
                          cudaStream_t s) {
  const int64_t total = n * ncomp;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = unsigned((total + threads - 1) / threads);
  if (precision == ELM_FP64)
    k_gather<double><<<blocks, threads, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out), idx, n, ncomp);
  else
    k_gather<float><<<blocks, threads, 0, s>>>(static_cast<const float*>(in), static_cast<float*>(out), idx, n, ncomp);
  return cudaGetLastError();
}

}  // namespace elm
