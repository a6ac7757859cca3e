// tracer.cuh -- device code shared by the advection kernels (advect.cu) and
// their adjoint (adjoint.cu): point representation, macro walk, micro
// location, P2 stencils and the per-node forward step.  See advect.cu for
// the method and the GB300 design notes.
#pragma once

#include <cstdint>
#include <cfloat>
#include <type_traits>

#include "elm_internal.h"

namespace elm {
namespace {


constexpr double kTol64 = 1e-9;     // "inside" tolerance, lattice units (FP64)
constexpr float kBand32 = 3e-5f;    // FP32 tie band re-decided in FP64, lattice units

// ---------------------------------------------------------------------------
// Conversions of integer-valued lattice coordinates (exact for |v| < 2^22).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int f2i_exact(float x) { return __float2int_rn(x); }
__device__ __forceinline__ float i2f_exact(int i) { return __int2float_rn(i); }
// The FP64 forms below run on the integer pipe: this GPU's FP64 pipe (2
// lanes per SM and cycle) bounds the FP64 kernels, while their integer pipe
// idles.  Each gives the FP64 instruction's result on the operands it meets.
// Cell index of an integer-valued double 0 <= x < 2^21 (a located cell),
// read from its exponent and leading mantissa bits.
// (Anything else, NaN included, gives an index in [0, 2^21).)
__device__ __forceinline__ int f2i_exact(double x) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) - 1023;  // x = +0: e < 0
  return (e < 0 || e > 20) ? 0 : (((hi & 0xFFFFF) | 0x100000) >> (20 - e));
}
__device__ __forceinline__ double i2f_exact_d(int i) {
  return __longlong_as_double(0x4338000000000000LL + i) - 6755399441055744.0;
}
template <class R>
__device__ __forceinline__ R to_real(int i);
template <>
__device__ __forceinline__ float to_real<float>(int i) { return i2f_exact(i); }
template <>
__device__ __forceinline__ double to_real<double>(int i) { return i2f_exact_d(i); }

// floor for |x| < 2^22 on the FMA pipe: adding 1.5 * 2^23 rounds x to the
// nearest integer, which is then corrected down if it lies above x.
__device__ __forceinline__ float floor_small(float x) {
  const float r = (x + 12582912.0f) - 12582912.0f;
  return r > x ? r - 1.0f : r;
}

// Precision-exact math: the float overloads never promote to FP64.
__device__ __forceinline__ float r_floor(float x) { return floorf(x); }
// floor of a finite double by clearing its fraction bits (one FP64
// subtraction only for negative non-integers).
__device__ __forceinline__ double r_floor(double x) {
  const long long b = __double_as_longlong(x);
  const int e = int((b >> 52) & 0x7FF) - 1023;
  if (e >= 52) return x;                                           // integer already
  if (e < 0) return b < 0 ? ((b << 1) == 0 ? x : -1.0) : 0.0;      // |x| < 1 (floor(-0) = -0)
  const long long frac = (1LL << (52 - e)) - 1;
  if ((b & frac) == 0) return x;
  const double t = __longlong_as_double(b & ~frac);                // trunc(x)
  return b < 0 ? t - 1.0 : t;
}
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float r_clamp(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }
__device__ __forceinline__ float r_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double r_min(double a, double b) { return ::fmin(a, b); }
// Order-preserving integer image of a double that is not NaN: x < y exactly
// when d_key(x) < d_key(y) (-0 just below +0).
__device__ __forceinline__ long long d_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
// clamp(x, lo, hi) for lo <= hi by integer compares; like fmin(fmax(x, lo),
// hi) it returns a bound, never NaN, for a NaN x.
__device__ __forceinline__ double r_clamp(double x, double lo, double hi) {
  const long long k = d_key(x);
  if (k < d_key(lo)) return lo;
  return k > d_key(hi) ? hi : x;
}
// a > b and a >= b for doubles that are not NaN, by integer compares.  The
// location only meets finite values: every point it is given has passed the
// clamp, which maps a NaN or infinite coordinate to a bound.
__device__ __forceinline__ bool r_greater(double a, double b) { return d_key(a) > d_key(b); }
__device__ __forceinline__ bool r_greater(float a, float b) { return a > b; }
__device__ __forceinline__ bool r_geq(double a, double b) { return d_key(a) >= d_key(b); }
__device__ __forceinline__ bool r_geq(float a, float b) { return a >= b; }

// ---------------------------------------------------------------------------
// Double-float helpers (error-free transformations; no FP64 instructions).
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_renorm(float s, float e) {
  const float hi = s + e;
  return {hi, e - (hi - s)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  return df_renorm(s, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
  return df_renorm(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.hi, b, -p) + a.lo * b;
  return df_renorm(p, e);
}

// ---------------------------------------------------------------------------
// Macro tables in the working precision.
// ---------------------------------------------------------------------------
template <class R>
struct Tables;

template <>
struct Tables<double> {
  const MacroGeo* g;
  __device__ double nj(int m, int k) const { return g[m].NJinv[k]; }
  __device__ double J(int m, int k) const { return g[m].J[k]; }
  __device__ double v0(int m, int k) const { return g[m].v0[k]; }
  __device__ int nb(int m, int k) const { return g[m].nb[k]; }
  __device__ const FaceXform& xf(int m) const { return g[m].x; }
};

template <>
struct Tables<float> {
  const MacroGeo32* g;
  __device__ float nj(int m, int k) const { return g[m].NJinv[k]; }
  __device__ float J(int m, int k) const { return g[m].J[k]; }
  __device__ float v0(int m, int k) const { return g[m].v0[k]; }
  __device__ int nb(int m, int k) const { return g[m].nb[k]; }
  __device__ const FaceXform& xf(int m) const { return g[m].x; }
};

__device__ __forceinline__ int tri2(int k) { return k * (k + 1) / 2; }
__device__ __forceinline__ int tri3(int k) { return k * (k + 1) * (k + 2) / 6; }

// Slot within a macro -> lattice point p (packed order p1, p2[, p3]).  The
// row and slab are estimated with the MUFU log2/exp2/rsqrt approximations
// (cbrt(6 r), (sqrt(8 r + 1) - 1) / 2) and made exact by integer fix-up
// loops; libm's cbrtf/sqrtf would add FP64 or long FP32 sequences.

template <int D>
__device__ __forceinline__ int tri_root2(int r) {
  const float x = 8.0f * i2f_exact(r) + 1.0f;
  int k = f2i_exact(floor_small((x * rsqrtf(x) - 1.0f) * 0.5f));
  k = max(k, 0);
  while (k > 0 && tri2(k) > r) --k;
  while (tri2(k + 1) <= r) ++k;
  return k;
}

// ---------------------------------------------------------------------------
// Rare paths: entering a foreign macro and the FP64 tie-break.  They are free,
// non-inlined functions taking scalars and returning small structs: the
// start-node position they need is loop-invariant, and once inlined the
// compiler hoists that FP64 / double-float work out of the rare branch into
// every thread (costly on this GPU's narrow FP64 pipe), while a non-inlined
// member function would force the tracer state onto the stack.
// ---------------------------------------------------------------------------
struct Frame {
  float bq0, bq1, bq2, r00, r01, r02;
};
struct FrameD {
  double bq0, bq1, bq2, r00, r01, r02;
};
struct Min64 {
  double lmin;
  int kmin;
};

// Start node x_i = v0_m0 + J_m0 (p / M) in FP64; the node lattice has
// M = P N points per macro edge (P2: vertices and midpoints, P1: vertices).
template <int D, int P>
__device__ __forceinline__ void node_position64(const MacroGeo* geo, int m0, int p0, int p1, int p2, int N,
                                                double* x) {
  const MacroGeo& g0 = geo[m0];
  // 1 / M, M = 2^k: the exponent field set directly (an FP64 division would
  // take dozens of instructions on the narrow FP64 pipe)
  const double invM = __longlong_as_double(static_cast<long long>(1024 - __ffs(P * N)) << 52);
  const double s[3] = {double(p0) * invM, double(p1) * invM, double(p2) * invM};
#pragma unroll
  for (int r = 0; r < D; ++r) {
    double v = g0.v0[r];
#pragma unroll
    for (int c = 0; c < D; ++c) v = ::fma(g0.J[r * 3 + c], s[c], v);
    x[r] = v;
  }
}

// Lattice coordinate of the start node in macro mm, FP64.
template <int D, int P>
__device__ __forceinline__ void node_lattice64(const MacroGeo* geo, int m0, int p0, int p1, int p2, int N, int mm,
                                               double* q) {
  double x[D];
  node_position64<D, P>(geo, m0, p0, p1, p2, N, x);
  const MacroGeo& g = geo[mm];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) v = ::fma(g.NJinv[r * 3 + c], x[c] - g.v0[c], v);
    q[r] = v;
  }
}

template <int D, int P>
__device__ __noinline__ FrameD frame64(const MacroGeo* geo, int m0, int p0, int p1, int p2, int N, int mm) {
  double q[3] = {0.0, 0.0, 0.0};
  node_lattice64<D, P>(geo, m0, p0, p1, p2, N, mm, q);
  FrameD f;
  f.bq0 = ::floor(q[0]);
  f.bq1 = ::floor(q[1]);
  f.bq2 = ::floor(q[2]);
  f.r00 = q[0] - f.bq0;
  f.r01 = q[1] - f.bq1;
  f.r02 = q[2] - f.bq2;
  return f;
}

// double-float on the FP32 pipe: x_i = v0_m0 + J_m0 (p / M); q = NJinv_mm (x_i - v0_mm)
template <int D>
__device__ __noinline__ Frame frame_df(const MacroGeo32* tg, int m0, int p0, int p1, int p2, float invM, int mm) {
  const MacroGeo32& g0 = tg[m0];
  const MacroGeo32& g = tg[mm];
  const int pp[3] = {p0, p1, p2};
  df y[D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    df acc = {g0.v0[r], g0.v0_lo[r]};
#pragma unroll
    for (int c = 0; c < D; ++c)
      acc = df_add(acc, df_mul_f(df{g0.J[r * 3 + c], g0.J_lo[r * 3 + c]}, i2f_exact(pp[c]) * invM));
    y[r] = df_add(acc, df{-g.v0[r], -g.v0_lo[r]});
  }
  float bq[3] = {0.0f, 0.0f, 0.0f}, r0[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int r = 0; r < D; ++r) {
    df q = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < D; ++c) q = df_add(q, df_mul(df{g.NJinv[r * 3 + c], g.NJinv_lo[r * 3 + c]}, y[c]));
    float fl = floor_small(q.hi);
    if (fl == q.hi && q.lo < 0.0f) fl -= 1.0f;
    bq[r] = fl;
    r0[r] = (q.hi - fl) + q.lo;
  }
  return Frame{bq[0], bq[1], bq[2], r0[0], r0[1], r0[2]};
}

// FP64 minimum barycentric (lattice units) of x_i + d in macro m, and its face.
template <int D, int P>
__device__ __noinline__ Min64 bary64_min(const MacroGeo* geo, int m0, int p0, int p1, int p2, int N, int m,
                                         float d0, float d1, float d2) {
  double q[3] = {0.0, 0.0, 0.0};
  node_lattice64<D, P>(geo, m0, p0, p1, p2, N, m, q);
  const MacroGeo& g = geo[m];
  const double d[3] = {double(d0), double(d1), double(d2)};
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) q[r] = ::fma(g.NJinv[r * 3 + c], d[c], q[r]);
  double l[D + 1];
  l[0] = double(N) - q[0];
#pragma unroll
  for (int k = 1; k < D; ++k) l[k] = q[k - 1] - q[k];
  l[D] = q[D - 1];
  Min64 out{l[0], 0};
#pragma unroll
  for (int k = 1; k <= D; ++k)
    if (l[k] < out.lmin) {
      out.lmin = l[k];
      out.kmin = k;
    }
  return out;
}

// The same minimum barycentric (lattice units) and face in double-float
// arithmetic on the FP32 pipe (about 44 significant bits: the lattice
// coordinate is exact to about 256 * 2^-44 = 1.5e-11, far inside the FP64
// decision's 1e-9 band).  Used by the trace and evaluation kernels, whose
// points can stay on an interior face for the whole trace (a flow that keeps
// a face invariant sends every lookup of those nodes here): their tie
// decisions then cost FP32 instructions instead of this part's narrow FP64
// pipe.  Ties of the minimum keep the lowest face index, like bary64_min.
template <int D>
__device__ __noinline__ Min64 bary_df_min(const MacroGeo32* tg, int m0, int p0, int p1, int p2, float invM, int m,
                                          float Nf, float d0, float d1, float d2) {
  const MacroGeo32& g0 = tg[m0];
  const MacroGeo32& g = tg[m];
  const int pp[3] = {p0, p1, p2};
  const float dd[3] = {d0, d1, d2};
  df y[D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    df acc = {g0.v0[r], g0.v0_lo[r]};
#pragma unroll
    for (int c = 0; c < D; ++c)
      acc = df_add(acc, df_mul_f(df{g0.J[r * 3 + c], g0.J_lo[r * 3 + c]}, i2f_exact(pp[c]) * invM));
    acc = df_add(acc, df{dd[r], 0.0f});
    y[r] = df_add(acc, df{-g.v0[r], -g.v0_lo[r]});
  }
  df q[D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    q[r] = df{0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < D; ++c) q[r] = df_add(q[r], df_mul(df{g.NJinv[r * 3 + c], g.NJinv_lo[r * 3 + c]}, y[c]));
  }
  df l[D + 1];
  l[0] = df_add(df{Nf, 0.0f}, df{-q[0].hi, -q[0].lo});
#pragma unroll
  for (int k = 1; k < D; ++k) l[k] = df_add(q[k - 1], df{-q[k].hi, -q[k].lo});
  l[D] = q[D - 1];
  Min64 out{0.0, 0};
  df best = l[0];
#pragma unroll
  for (int k = 1; k <= D; ++k)
    if (l[k].hi < best.hi || (l[k].hi == best.hi && l[k].lo < best.lo)) {
      best = l[k];
      out.kmin = k;
    }
  out.lmin = double(best.hi + best.lo);
  return out;
}

// Brute-force macro search for x_i + d (rare path): the macro whose reference
// simplex holds the point best (largest minimum barycentric, lattice units).
// On a non-convex mesh (an annulus) the walk can end at a boundary face while
// the point lies in the mesh behind it.
template <int D, class R, int P>
__device__ __noinline__ int best_macro(Tables<R> tab, const MacroGeo* geo, int nmac, int m0, int p0, int p1, int p2,
                                       int N, float invM, R d0, R d1, R d2) {
  const R d[3] = {d0, d1, d2};
  int best = m0;
  R bestl = R(-1e30);
  for (int mm = 0; mm < nmac; ++mm) {
    R bq[3], r0[3];
    if constexpr (sizeof(R) == 8) {
      const FrameD f = frame64<D, P>(geo, m0, p0, p1, p2, N, mm);
      bq[0] = f.bq0; bq[1] = f.bq1; bq[2] = f.bq2;
      r0[0] = f.r00; r0[1] = f.r01; r0[2] = f.r02;
    } else {
      const Frame f = frame_df<D>(tab.g, m0, p0, p1, p2, invM, mm);
      bq[0] = f.bq0; bq[1] = f.bq1; bq[2] = f.bq2;
      r0[0] = f.r00; r0[1] = f.r01; r0[2] = f.r02;
    }
    R q[3];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      R v = r0[k];
#pragma unroll
      for (int j = 0; j < D; ++j) v = r_fma(tab.nj(mm, k * 3 + j), d[j], v);
      q[k] = bq[k] + v;
    }
    R l = R(N) - q[0];
#pragma unroll
    for (int k = 1; k < D; ++k) l = r_min(l, q[k - 1] - q[k]);
    l = r_min(l, q[D - 1]);
    if (l > bestl) {
      bestl = l;
      best = mm;
    }
  }
  return best;
}

// r = r0 + N J_m^{-1} d in a macro other than the block's (after a hand-off;
// not inlined so the common path carries no table loads or selects).
template <class R>
struct Vec3 {
  R x, y, z;
};
template <int D, class R>
__device__ __noinline__ Vec3<R> lattice_foreign(Tables<R> tab, int m, R r00, R r01, R r02, R d0, R d1, R d2) {
  const R r0[3] = {r00, r01, r02};
  const R d[3] = {d0, d1, d2};
  R r[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    R v = r0[k];
#pragma unroll
    for (int j = 0; j < D; ++j) v = r_fma(tab.nj(m, k * 3 + j), d[j], v);
    r[k] = v;
  }
  return Vec3<R>{r[0], r[1], r[2]};
}

// Blending onto an annulus (Sec. 2.1; 2D, FP64).  The ring mesh's sector k
// (between the rays at theta_k = theta0 + k delta) holds the computational
// points x = rho ((1 - lam) e_k + lam e_{k+1}), rho between the chords of two
// circles; Phi(x) = rho e(theta_k + lam delta) carries chords onto arcs with
// uniform angle.  Phi^{-1}(y): lam from the polar angle of y, rho = |y|.
__device__ __noinline__ void blend_inv(const BlendArgs& b, double y0, double y1, double* xc) {
  const double t = (atan2(y1, y0) - b.theta0) / b.delta;
  const double kf = floor(t);
  const double lam = t - kf;
  int k = int(kf) % b.nsec;
  if (k < 0) k += b.nsec;
  const double rho = sqrt(y0 * y0 + y1 * y1);
  xc[0] = rho * ((1.0 - lam) * b.sec[2 * k] + lam * b.sec[2 * k + 2]);
  xc[1] = rho * ((1.0 - lam) * b.sec[2 * k + 1] + lam * b.sec[2 * k + 3]);
}

__device__ __noinline__ void blend_fwd(const BlendArgs& b, double x0, double x1, double* xp) {
  const double t = (atan2(x1, x0) - b.theta0) / b.delta;
  int k = int(floor(t)) % b.nsec;
  if (k < 0) k += b.nsec;
  const double e0 = b.sec[2 * k], e1 = b.sec[2 * k + 1], f0 = b.sec[2 * k + 2], f1 = b.sec[2 * k + 3];
  // x parallel to (1 - lam) e_k + lam e_{k+1}
  const double ck = e0 * x1 - e1 * x0, ck1 = f0 * x1 - f1 * x0;
  const double lam = ck / (ck - ck1);
  const double p0 = (1.0 - lam) * e0 + lam * f0, p1 = (1.0 - lam) * e1 + lam * f1;
  const double rho = sqrt(x0 * x0 + x1 * x1) / sqrt(p0 * p0 + p1 * p1);
  double s, c;
  sincos(b.theta0 + (double(k) + lam) * b.delta, &s, &c);
  xp[0] = rho * c;
  xp[1] = rho * s;
}

// Per-thread tracing state.  P is the element order of the velocity and the
// scalar (Sec. 3.1: linear P1 or quadratic P2 Lagrange elements).  BLEND = 1:
// the mesh is blended onto an annulus; points and offsets are physical and
// pulled back with Phi^{-1} before location.
// Start-node state of the blended form (empty otherwise).
struct BlendState {
  BlendArgs bl;
  double xc[2], xp[2];  // start node: computational and physical position
};
struct NoBlendState {};

// Kuhn ordering of the cell fractions f (descending, ties by axis): sigma0
// and sigma1, the sorted fractions fs0 >= fs1 >= fs2, and the P2 basis values
// of the micro simplex's vertices (v0..v3) and edges (01 02 03 12 13 23).
struct KuhnP2 {
  bool first0, first1;  // sigma0 = 0, sigma0 = 1 (else 2)
  bool sec2, sec1;      // sigma1 = 2, sigma1 = 1 (else 0)
};
template <class R>
__device__ __forceinline__ KuhnP2 kuhn_p2_3d(const R* f, R* phi) {
  KuhnP2 o;
  const bool g01 = f[1] > f[0], g02 = f[2] > f[0], g12 = f[2] > f[1];
  o.first0 = !g01 && !g02;
  o.first1 = !o.first0 && !g12;
  o.sec2 = o.first0 ? g12 : (o.first1 ? g02 : false);
  o.sec1 = o.first0 ? !g12 : (o.first1 ? false : g01);
  const R fs0 = o.first0 ? f[0] : (o.first1 ? f[1] : f[2]);
  const R fs1 = o.sec2 ? f[2] : (o.sec1 ? f[1] : f[0]);
  const R fs2 = r_min(r_min(f[0], f[1]), f[2]);
  const R L0 = R(1) - fs0, L1 = fs0 - fs1, L2 = fs1 - fs2, L3 = fs2;
  phi[0] = L0 * (R(2) * L0 - R(1));
  phi[1] = L1 * (R(2) * L1 - R(1));
  phi[2] = L2 * (R(2) * L2 - R(1));
  phi[3] = L3 * (R(2) * L3 - R(1));
  phi[4] = R(4) * L0 * L1;
  phi[5] = R(4) * L0 * L2;
  phi[6] = R(4) * L0 * L3;
  phi[7] = R(4) * L1 * L2;
  phi[8] = R(4) * L1 * L3;
  phi[9] = R(4) * L2 * L3;
  return o;
}

// TIE_DF (FP32 only): interior-face tie decisions in double-float on the FP32
// pipe (bary_df_min) instead of FP64 (bary64_min); the trace and evaluation
// kernels use it, the step kernel keeps the FP64 decision.
template <int D, class R, bool STEADY, int P = 2, int BLEND = 0, int TIE_DF = 0>
struct Tracer : std::conditional_t<BLEND == 1, BlendState, NoBlendState> {
  static_assert(BLEND == 0 || (D == 2 && sizeof(R) == 8), "blending: 2D FP64 only");
  static_assert(P == 1 || P == 2, "element order");
  static_assert(TIE_DF == 0 || sizeof(R) == 4, "double-float tie decisions serve the FP32 kernels");
  static constexpr int NB = P == 2 ? (D + 1) * (D + 2) / 2 : D + 1;  // nodes of a simplex
  // launch constants (copied, so no kernel parameter is addressed)
  const MacroGeo* geo;   // FP64 macro table (tie-breaks)
  Tables<R> tab;         // macro table in the working precision
  int N;
  int npm;
  int nmac = 0;    // macros of the mesh (0: no brute-force search)
  const R* un;
  const R* uo;
  const R* T;
  R dt;
  R Nf;
  R invM;          // 1 / M, M = P 2^L (node lattice), exact
  unsigned* status;
  int m0;          // home macro
  int p[D];        // home lattice point
  // current frame: q = bq + r0 + nj * d
  int m;
  R bq[D];
  R r0[D];
  int mb;             // the block's macro (uniform across the block)
  R njb[D * D];       // N J^{-1} of the block's macro
  R bo[D + 1];        // per face of the block's macro: the tie band (interior face) or 0 (boundary face)
  R dlo[D], dhi[D];  // box limits as offsets from x_i

  static constexpr R kBand = sizeof(R) == 4 ? R(kBand32) : R(kTol64);

  __device__ void load_block_macro(int mm) {
    mb = mm;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) njb[r * D + c] = tab.nj(mm, r * 3 + c);
    // A point within the band of a boundary face needs no walk decision (there
    // is no macro behind it), so only interior faces keep the band.
#pragma unroll
    for (int k = 0; k <= D; ++k) bo[k] = tab.nb(mm, k) >= 0 ? kBand : R(0);
  }

  // Retraction into the reference simplex N >= q1 >= q2 (>= q3) >= 0: the
  // cell is clamped to [0, N-1] and the order of the axes restored.
  __device__ void retract(R* c, R* f) const {
    if (c[0] < R(0)) { c[0] = R(0); f[0] = R(0); }
    if (c[0] > Nf - R(1)) { c[0] = Nf - R(1); f[0] = R(1); }
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (c[k] > c[k - 1] || (c[k] == c[k - 1] && f[k] > f[k - 1])) { c[k] = c[k - 1]; f[k] = f[k - 1]; }
      if (c[k] < R(0)) { c[k] = R(0); f[k] = R(0); }
    }
  }

  // N J^{-1} entry of the current macro: the block's macro from registers,
  // any other (after a hand-off) from the L1-resident table.
  __device__ R nj(int k) const { return m == mb ? njb[k] : tab.nj(m, (k / D) * 3 + k % D); }

  __device__ void home_frame() {
    m = m0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (P == 2) {
        bq[k] = to_real<R>(p[k] >> 1);
        r0[k] = (p[k] & 1) ? R(0.5) : R(0);
      } else {
        bq[k] = to_real<R>(p[k]);
        r0[k] = R(0);
      }
    }
  }

  // Enters macro mm: (bq, r0) of the start node in mm's frame.
  __device__ void foreign_frame(int mm) {
    if (mm == m0) {
      home_frame();
      return;
    }
    m = mm;
    if constexpr (sizeof(R) == 8) {
      const FrameD f = frame64<D, P>(geo, m0, p[0], p[1], D == 3 ? p[D - 1] : 0, N, mm);
      bq[0] = f.bq0;
      bq[1] = f.bq1;
      r0[0] = f.r00;
      r0[1] = f.r01;
      if (D == 3) {
        bq[D - 1] = f.bq2;
        r0[D - 1] = f.r02;
      }
    } else {
      const Frame f = frame_df<D>(tab.g, m0, p[0], p[1], D == 3 ? p[D - 1] : 0, float(invM), mm);
      bq[0] = R(f.bq0);
      bq[1] = R(f.bq1);
      r0[0] = R(f.r00);
      r0[1] = R(f.r01);
      if (D == 3) {
        bq[D - 1] = R(f.bq2);
        r0[D - 1] = R(f.r02);
      }
    }
  }

  // Walks across face k of the current macro into its neighbour mm.  Across a
  // face with an exact integer frame change (FaceXform) a start node on the
  // half-integer lattice of the current frame changes frame exactly in the
  // working precision (a few FMAs); otherwise the frame is recomputed from
  // the start node (foreign_frame).  Both give the same (bq, r0).
  __device__ void cross_face(int mm, int k) {
    if (mm != m0) {
      const FaceXform& x = tab.xf(m);
      bool half = ((x.exact >> k) & 1) != 0;
#pragma unroll
      for (int j = 0; j < D; ++j) half = half && (r0[j] == R(0) || r0[j] == R(0.5));
      if (half) {
        R s[D], q[D];
#pragma unroll
        for (int j = 0; j < D; ++j) s[j] = bq[j] + r0[j];
#pragma unroll
        for (int r = 0; r < D; ++r) {
          R v = to_real<R>(x.b[k][r]);
#pragma unroll
          for (int c = 0; c < D; ++c) v = r_fma(to_real<R>(x.A[k][r * 3 + c]), s[c], v);
          q[r] = v;
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
          const R fl = r_floor(q[r]);
          bq[r] = fl;
          r0[r] = q[r] - fl;
        }
        m = mm;
        return;
      }
    }
    foreign_frame(mm);
  }

  // Locates x_i + d: walks macros from the current frame, returns the micro
  // cell c (integer-valued reals) and fractions f, retracted into the
  // macro's reference simplex N >= q1 >= q2 (>= q3) >= 0.
  __device__ void locate(const R* d, R* c, R* f) {
    R lmin;
    bool searched = false;
    for (int hop = 0;; ++hop) {
      R r[D];
      if (m == mb) {
        if constexpr (sizeof(R) == 4 && D == 3) {
          // rows 0 and 1 as one packed FP32x2 FMA chain (same per-lane rounding)
          float2 a01 = make_float2(r0[0], r0[1]);
          float a2 = r0[D - 1];
#pragma unroll
          for (int j = 0; j < D; ++j) {
            a01 = __ffma2_rn(make_float2(njb[j], njb[D + j]), make_float2(d[j], d[j]), a01);
            a2 = fmaf(njb[2 * D + j], d[j], a2);
          }
          r[0] = a01.x;
          r[1] = a01.y;
          r[D - 1] = a2;
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            R v = r0[k];
#pragma unroll
            for (int j = 0; j < D; ++j) v = r_fma(njb[k * D + j], d[j], v);
            r[k] = v;
          }
        }
      } else {
        const Vec3<R> v = lattice_foreign<D, R>(tab, m, r0[0], r0[1], D == 3 ? r0[D - 1] : R(0), d[0], d[1],
                                                D == 3 ? d[D - 1] : R(0));
        r[0] = v.x;
        r[1] = v.y;
        if (D == 3) r[D - 1] = v.z;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const R fl = r_floor(r[k]);
        c[k] = bq[k] + fl;
        f[k] = r[k] - fl;
      }
      R l[D + 1];
      l[0] = (Nf - c[0]) - f[0];
#pragma unroll
      for (int k = 1; k < D; ++k) l[k] = (c[k - 1] - c[k]) + (f[k - 1] - f[k]);
      l[D] = c[D - 1] + f[D - 1];
      // common case: inside the block's macro, clear of its interior faces.
      // With every l >= 0 the cell is in range except on the face q1 = N
      // (c1 = N) and where a tiny negative r (|r| below half an ulp of 1)
      // made f = r - floor(r) round up to 1 with c = -1 in the last axis
      // (l_d = c + f = 0 hides it); the retraction clamps both.
      {
        bool in = m == mb;
#pragma unroll
        for (int k = 0; k <= D; ++k) in = in && r_geq(l[k], bo[k]);
        if (in) {
          if (r_greater(c[0], Nf - R(1)) || r_greater(R(0), c[D - 1])) retract(c, f);
          return;
        }
      }
      lmin = l[0];
#pragma unroll
      for (int k = 1; k <= D; ++k) lmin = r_min(lmin, l[k]);
      // a foreign macro, clear of its faces
      if (lmin >= kBand) return;
      int kmin = D;
#pragma unroll
      for (int k = D - 1; k >= 0; --k)
        if (l[k] == lmin) kmin = k;
      bool outside;
      int nb;
      if constexpr (sizeof(R) == 4) {
        outside = lmin < R(-kBand32);
        nb = tab.nb(m, kmin);
        if (!outside && nb >= 0) {
          // tie band at an interior face: decide in FP64 from the exact start node
          Min64 r64;
          if constexpr (TIE_DF == 1)
            r64 = bary_df_min<D>(tab.g, m0, p[0], p[1], D == 3 ? p[D - 1] : 0, float(invM), m, float(Nf),
                                 float(d[0]), float(d[1]), D == 3 ? float(d[D - 1]) : 0.0f);
          else
            r64 = bary64_min<D, P>(geo, m0, p[0], p[1], D == 3 ? p[D - 1] : 0, N, m, float(d[0]), float(d[1]),
                                   D == 3 ? float(d[D - 1]) : 0.0f);
          outside = r64.lmin < -kTol64;
          kmin = r64.kmin;
          nb = tab.nb(m, kmin);
        }
      } else {
        outside = lmin < R(-kTol64);
        nb = outside ? tab.nb(m, kmin) : -1;
      }
      if constexpr (BLEND == 1) {
        if (outside && nb < 0) {
          // The most negative face is a boundary face.  On the non-convex
          // annulus the point can still lie in the mesh behind another
          // negative face: walk across the most negative face that has a
          // neighbour, if any.  (Box domains are convex: a clamped point is
          // never outside through a boundary face beyond the band.)
          R best = -kBand;
#pragma unroll
          for (int k = 0; k <= D; ++k) {
            if (l[k] < best) {
              const int n2 = tab.nb(m, k);
              if (n2 >= 0) {
                best = l[k];
                kmin = k;
                nb = n2;
              }
            }
          }
        }
        if (outside && nb < 0 && nmac > 0 && !searched) {
          // still outside only through boundary faces of a non-convex mesh:
          // search every macro once
          searched = true;
          const int mm = best_macro<D, R, P>(tab, geo, nmac, m0, p[0], p[1], D == 3 ? p[D - 1] : 0, N,
                                             float(invM), d[0], d[1], D == 3 ? d[D - 1] : R(0));
          if (mm != m) {
            foreign_frame(mm);
            continue;
          }
        }
      }
      if (!outside || nb < 0) break;  // inside, or outside the mesh (retraction clamps)
      if (hop >= kMaxHops) {
        atomicOr(status, kFlagWalkLimit);
        break;
      }
      cross_face(nb, kmin);
    }
    if (lmin > R(0)) return;
    retract(c, f);
  }

  // P2 stencil of the micro simplex holding (c, f): storage slots and basis
  // values (the macro's base slot is folded into the last axis' table).  Per axis a the packed index contributes A_a[o] for the
  // lattice offset o in {0, 1, 2} of the node from 2c; sorting the axes by
  // descending fraction (ties by axis) orders the Kuhn path c -> c + 1, and
  // each node's offsets along the sorted axes are fixed (alpha >= beta >= gamma).
  // 3D P2 stencil by ranks (FP32 kernel): the packed index of c + o is S0
  // plus per-axis increments (T3 / T2 differences for the first two axes, 1
  // and 2 for the last), so with the axes in stable descending order of their
  // fractions (sigma0, sigma1, sigma2) only the increments of sigma0 and
  // sigma1 are selected, and the all-1 and all-2 offsets need no order.  Same
  // slots and basis values as the sorting form below, with fewer selects;
  // sigma0 != sigma1 by construction, so the slots are always those of a
  // valid micro simplex.  (The FP64 kernel keeps the sorting form: its extra
  // FP64 min operations would load the narrow FP64 pipe.)
  __device__ void stencil_p2_3d(const R* c, const R* f, int* slot, R* phi) const {
    static_assert(NB == 10, "3D P2 stencil");
    const int k0 = 2 * f2i_exact(c[0]);
    const int k1 = 2 * f2i_exact(c[1]);
    const int k2 = 2 * f2i_exact(c[2]);
    const int d10 = tri2(k0 + 1);          // T3(k0 + 1) - T3(k0)
    const int d20 = d10 + tri2(k0 + 2);    // T3(k0 + 2) - T3(k0)
    const int d11 = k1 + 1;                // T2(k1 + 1) - T2(k1)
    const int d21 = 2 * k1 + 3;            // T2(k1 + 2) - T2(k1)
    const int S0 = tri3(k0) + tri2(k1) + k2 + m * npm;
    const int S1 = S0 + d10 + d11 + 1;
    const int S2 = S0 + d20 + d21 + 2;
    const KuhnP2 o = kuhn_p2_3d(f, phi);
    const bool first0 = o.first0, first1 = o.first1, sec2 = o.sec2, sec1 = o.sec1;
    const int a1 = first0 ? d10 : (first1 ? d11 : 1);
    const int a2 = first0 ? d20 : (first1 ? d21 : 2);
    const int b1 = sec2 ? 1 : (sec1 ? d11 : d10);
    const int b2 = sec2 ? 2 : (sec1 ? d21 : d20);
    const int v1 = S0 + a2;
    const int e01 = S0 + a1;
    const int e13 = S1 + a2 - a1;
    slot[0] = S0;
    slot[1] = v1;
    slot[2] = v1 + b2;
    slot[3] = S2;
    slot[4] = e01;
    slot[5] = e01 + b1;
    slot[6] = S1;
    slot[7] = v1 + b1;
    slot[8] = e13;
    slot[9] = e13 + b2 - b1;
  }

  __device__ void stencil(const R* c, const R* f, int* slot, R* phi) const {
    if constexpr (P == 1) {
      stencil_p1(c, f, slot, phi);
      return;
    }
    if constexpr (P == 2 && D == 3 && sizeof(R) == 4) {
      stencil_p2_3d(c, f, slot, phi);
      return;
    }
    int A[D][3];
    R fs[D];
    {
      const int base = m * npm;  // the macro's first storage slot (storage < 2^31)
      const int c0 = 2 * f2i_exact(c[0]);
      if (D == 3) {
        const int c1 = 2 * f2i_exact(c[1]);
        const int c2 = 2 * f2i_exact(c[D - 1]) + base;
        A[0][0] = tri3(c0);
        A[0][1] = A[0][0] + tri2(c0 + 1);
        A[0][2] = A[0][1] + tri2(c0 + 2);
        A[1][0] = tri2(c1);
        A[1][1] = A[1][0] + c1 + 1;
        A[1][2] = A[1][1] + c1 + 2;
        A[D - 1][0] = c2;
        A[D - 1][1] = c2 + 1;
        A[D - 1][2] = c2 + 2;
      } else {
        const int c1 = 2 * f2i_exact(c[D - 1]) + base;
        A[0][0] = tri2(c0);
        A[0][1] = A[0][0] + c0 + 1;
        A[0][2] = A[0][1] + c0 + 2;
        A[D - 1][0] = c1;
        A[D - 1][1] = c1 + 1;
        A[D - 1][2] = c1 + 2;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) fs[k] = f[k];
    }
    auto cswap = [&](int i, int j) {
      if (r_greater(fs[j], fs[i])) {
        R t = fs[i]; fs[i] = fs[j]; fs[j] = t;
#pragma unroll
        for (int o = 0; o < 3; ++o) { int u = A[i][o]; A[i][o] = A[j][o]; A[j][o] = u; }
      }
    };
    R L[D + 1];
    if (D == 3) {
      cswap(0, 1); cswap(1, 2); cswap(0, 1);
      L[0] = R(1) - fs[0];
      L[1] = fs[0] - fs[1];
      L[2] = fs[1] - fs[D - 1];
      L[D] = fs[D - 1];
      // vertices v0..v3, edges 01 02 03 12 13 23
      slot[0] = A[0][0] + A[1][0] + A[D - 1][0];
      slot[1] = A[0][2] + A[1][0] + A[D - 1][0];
      slot[2] = A[0][2] + A[1][2] + A[D - 1][0];
      slot[3] = A[0][2] + A[1][2] + A[D - 1][2];
      slot[4] = A[0][1] + A[1][0] + A[D - 1][0];
      slot[5] = A[0][1] + A[1][1] + A[D - 1][0];
      slot[6] = A[0][1] + A[1][1] + A[D - 1][1];
      slot[7] = A[0][2] + A[1][1] + A[D - 1][0];
      slot[8] = A[0][2] + A[1][1] + A[D - 1][1];
      slot[9 % NB] = A[0][2] + A[1][2] + A[D - 1][1];
      phi[0] = L[0] * (R(2) * L[0] - R(1));
      phi[1] = L[1] * (R(2) * L[1] - R(1));
      phi[2] = L[2] * (R(2) * L[2] - R(1));
      phi[3] = L[D] * (R(2) * L[D] - R(1));
      phi[4] = R(4) * L[0] * L[1];
      phi[5] = R(4) * L[0] * L[2];
      phi[6] = R(4) * L[0] * L[D];
      phi[7] = R(4) * L[1] * L[2];
      phi[8] = R(4) * L[1] * L[D];
      phi[9 % NB] = R(4) * L[2] * L[D];
    } else {
      cswap(0, 1);
      L[0] = R(1) - fs[0];
      L[1] = fs[0] - fs[D - 1];
      L[D] = fs[D - 1];
      // vertices v0..v2, edges 01 02 12
      slot[0] = A[0][0] + A[D - 1][0];
      slot[1] = A[0][2] + A[D - 1][0];
      slot[2] = A[0][2] + A[D - 1][2];
      slot[3] = A[0][1] + A[D - 1][0];
      slot[4] = A[0][1] + A[D - 1][1];
      slot[5] = A[0][2] + A[D - 1][1];
      phi[0] = L[0] * (R(2) * L[0] - R(1));
      phi[1] = L[1] * (R(2) * L[1] - R(1));
      phi[2] = L[D] * (R(2) * L[D] - R(1));
      phi[3] = R(4) * L[0] * L[1];
      phi[4] = R(4) * L[0] * L[D];
      phi[5] = R(4) * L[1] * L[D];
    }
  }

  // P1 stencil: the d+1 vertices of the micro simplex holding (c, f), whose
  // lattice points are c plus 0 or 1 per axis (node lattice = cell lattice),
  // with the micro barycentrics as basis values (Sec. 3.1, linear elements).
  // Per axis a the packed index contributes B_a[o], o in {0, 1}; sorting the
  // axes by descending fraction orders the Kuhn path c -> c + 1.
  __device__ void stencil_p1(const R* c, const R* f, int* slot, R* phi) const {
    int B[D][2];
    R fs[D];
    {
      const int base = m * npm;
      const int c0 = f2i_exact(c[0]);
      if (D == 3) {
        const int c1 = f2i_exact(c[1]);
        const int c2 = f2i_exact(c[D - 1]) + base;
        B[0][0] = tri3(c0);
        B[0][1] = B[0][0] + tri2(c0 + 1);
        B[1][0] = tri2(c1);
        B[1][1] = B[1][0] + c1 + 1;
        B[D - 1][0] = c2;
        B[D - 1][1] = c2 + 1;
      } else {
        const int c1 = f2i_exact(c[D - 1]) + base;
        B[0][0] = tri2(c0);
        B[0][1] = B[0][0] + c0 + 1;
        B[D - 1][0] = c1;
        B[D - 1][1] = c1 + 1;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) fs[k] = f[k];
    }
    auto cswap = [&](int i, int j) {
      if (r_greater(fs[j], fs[i])) {
        R t = fs[i]; fs[i] = fs[j]; fs[j] = t;
        int u0 = B[i][0]; B[i][0] = B[j][0]; B[j][0] = u0;
        int u1 = B[i][1]; B[i][1] = B[j][1]; B[j][1] = u1;
      }
    };
    if (D == 3) {
      cswap(0, 1); cswap(1, 2); cswap(0, 1);
      slot[0] = B[0][0] + B[1][0] + B[D - 1][0];
      slot[1] = B[0][1] + B[1][0] + B[D - 1][0];
      slot[2] = B[0][1] + B[1][1] + B[D - 1][0];
      slot[D] = B[0][1] + B[1][1] + B[D - 1][1];
      phi[0] = R(1) - fs[0];
      phi[1] = fs[0] - fs[1];
      phi[2] = fs[1] - fs[D - 1];
      phi[D] = fs[D - 1];
    } else {
      cswap(0, 1);
      slot[0] = B[0][0] + B[D - 1][0];
      slot[1] = B[0][1] + B[D - 1][0];
      slot[D] = B[0][1] + B[D - 1][1];
      phi[0] = R(1) - fs[0];
      phi[1] = fs[0] - fs[D - 1];
      phi[D] = fs[D - 1];
    }
  }

  __device__ void clamp_box(R* d) const {
    if constexpr (BLEND == 1) {
      // the annulus: radius clamped to [r_min, r_max] (Euclidean projection)
      const double y0 = this->xp[0] + d[0], y1 = this->xp[1] + d[1];
      const double r = sqrt(y0 * y0 + y1 * y1);
      if (!(r >= this->bl.rmin && r <= this->bl.rmax)) {
        if (r > 0.0 && r <= DBL_MAX) {
          const double s = fmin(fmax(r, this->bl.rmin), this->bl.rmax) / r;
          d[0] = s * y0 - this->xp[0];
          d[1] = s * y1 - this->xp[1];
        } else {
          // the centre, or a non-finite point (a NaN or infinite velocity):
          // the point (r_min, 0), so that no later location sees a NaN
          d[0] = this->bl.rmin - this->xp[0];
          d[1] = -this->xp[1];
        }
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) d[k] = r_clamp(d[k], dlo[k], dhi[k]);
  }

  // Offset in the coordinates the mesh is located in: d itself, or on a
  // blended mesh Phi^{-1}(x_i + d) - Phi^{-1}(x_i).
  __device__ void to_comp(const R* d, R* dc) const {
    if constexpr (BLEND == 1) {
      double yc[2];
      blend_inv(this->bl, this->xp[0] + d[0], this->xp[1] + d[1], yc);
      dc[0] = yc[0] - this->xc[0];
      dc[1] = yc[1] - this->xc[1];
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) dc[k] = d[k];
    }
  }

  // Velocity u~ at x_i + d at backward time `back` (Eq. linear interpolation).
  // Velocities are packed records (x, y[, z], 0): one vector load per node.
  __device__ void velocity(const R* d, R back, R* k) {
    R c[D], f[D];
    if constexpr (BLEND == 1) {
      R dc[D];
      to_comp(d, dc);
      locate(dc, c, f);
    } else {
      locate(d, c, f);
    }
    int slot[NB];
    R phi[NB];
    stencil(c, f, slot, phi);
    if constexpr (sizeof(R) == 4 && D == 3) {
      // (x, y) as one packed FP32x2 FMA chain (same per-lane rounding and order)
      float2 kxy = make_float2(0.f, 0.f);
      float kz = 0.f;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(un) + slot[j]);
        kxy = __ffma2_rn(make_float2(phi[j], phi[j]), make_float2(w.x, w.y), kxy);
        kz = fmaf(phi[j], w.z, kz);
      }
      k[0] = kxy.x;
      k[1] = kxy.y;
      k[D - 1] = kz;
    } else {
#pragma unroll
      for (int r = 0; r < D; ++r) k[r] = R(0);
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        R v[D];
        load_rec(un, slot[j], v);
#pragma unroll
        for (int r = 0; r < D; ++r) k[r] = r_fma(phi[j], v[r], k[r]);
      }
    }
    if constexpr (!STEADY) {
      R ko[D];
#pragma unroll
      for (int r = 0; r < D; ++r) ko[r] = R(0);
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        R v[D];
        load_rec(uo, slot[j], v);
#pragma unroll
        for (int r = 0; r < D; ++r) ko[r] = r_fma(phi[j], v[r], ko[r]);
      }
      const R w_old = back / dt, w_new = (dt - back) / dt;
#pragma unroll
      for (int r = 0; r < D; ++r) k[r] = w_old * ko[r] + w_new * k[r];
    }
  }

  // One packed velocity record.
  __device__ static void load_rec(const R* u, int node, R* v) {
    if constexpr (sizeof(R) == 4) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(u) + node);
      v[0] = w.x;
      v[1] = w.y;
      if (D == 3) v[D - 1] = w.z;
    } else {
      const double2 w = __ldg(reinterpret_cast<const double2*>(u) + 2 * node);
      v[0] = w.x;
      v[1] = w.y;
      if (D == 3) v[D - 1] = __ldg(u + 4 * int64_t(node) + 2);
    }
  }

  __device__ R scalar(const R* d) {
    R c[D], f[D];
    if constexpr (BLEND == 1) {
      R dc[D];
      to_comp(d, dc);
      locate(dc, c, f);
    } else {
      locate(d, c, f);
    }
    int slot[NB];
    R phi[NB];
    stencil(c, f, slot, phi);
    R v = R(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) v = r_fma(phi[j], __ldg(T + slot[j]), v);
    return v;
  }
};

// Resident 128-node chunks per SM (k_advect: 2 blocks of 64 threads each, so
// 16 blocks; 64 registers per thread): measured fastest on GB300 for the
// level-7 FP32 step (occupancy beats the few spills).
#ifndef ELM_ADVECT_MIN_BLOCKS
#define ELM_ADVECT_MIN_BLOCKS 8
#endif

template <class R>
__device__ __forceinline__ const StepConsts<R>& consts(const AdvectArgs& a);
template <>
__device__ __forceinline__ const StepConsts<float>& consts<float>(const AdvectArgs& a) { return a.k32; }
template <>
__device__ __forceinline__ const StepConsts<double>& consts<double>(const AdvectArgs& a) { return a.k64; }

template <int D>
__device__ __forceinline__ int packed(const int* p) {
  return D == 3 ? tri3(p[0]) + tri2(p[1]) + p[2] : tri2(p[0]) + p[1];
}

// Everything one node's step needs (one mesh instance, one call).
template <class R>
struct NodeJob {
  const MacroGeo* geo;
  const R* un;          // packed velocity records, u^{n+1}
  const R* uo;          // packed velocity records, u^n
  const R* T_old;
  R* T_new;
  unsigned* status;
  const int64_t* unique_map;
  const int64_t* owner_mp;
  StepConsts<R> K;
  int N;
  int npm;
  int n_sub;
  const R* D_in = nullptr;  // departure offsets [n, D] (trace / evaluation modes)
  R* D_out = nullptr;
  BlendArgs bl;             // annulus blending (BLEND = 1)
  int n_macros = 0;         // enables the brute-force search of non-convex meshes (BLEND = 1)
  int skip_ghosts = 0;      // copies held by a non-owner macro return at once (a copy pass fills them)
};

// What advect_node does with a node.
enum NodeMode {
  kStep = 0,   // trace from the node over dt, then T_new = T_old_h(X)  (steps (i)-(iii))
  kTrace = 1,  // continue the trace from x_i + D_in (or from x_i) over dt; D_out = X - x_i
  kEval = 2    // T_new = T_old_h(x_i + D_in)
};

// (ii) backward RK4 from x_i + d over dt: n_sub substeps of h = dt / n_sub.
// All 4 n_sub stage evaluations run through one loop with a single
// evaluation site (stage s of a substep sits at d, d - h/2 k, d - h/2 k,
// d - h k and has weight 1, 2, 2, 1), which keeps the kernel's code small.
// With from_node the first stage is the nodal value u_node (the P1 / P2
// interpolant at the node: steady, or at t_{n+1} where only u^{n+1} has
// weight).  Returns false if a stage combination was not finite.
template <int D, class R, class TR>
__device__ __forceinline__ bool rk4_backward(TR& t, const StepConsts<R>& K, int n_sub, const R* u_node,
                                             bool from_node, R* d) {
  const R h = K.h, h2 = K.h2, h6 = K.h6;
  bool finite = true;
  R k[D], acc[D];
#pragma unroll
  for (int q = 0; q < D; ++q) {
    k[q] = u_node[q];
    acc[q] = k[q];
  }
  const int n_eval = 4 * n_sub;
#pragma unroll 1
  for (int e = from_node ? 1 : 0; e < n_eval; ++e) {
    const int s = e & 3;
    const R off = s == 0 ? R(0) : (s == 3 ? h : h2);
    R z[D];
#pragma unroll
    for (int q = 0; q < D; ++q) z[q] = d[q] - off * k[q];
    t.clamp_box(z);
    t.velocity(z, to_real<R>(e >> 2) * h + off, k);
    const R w = (s == 1 || s == 2) ? R(2) : R(1);
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = s == 0 ? k[q] : r_fma(w, k[q], acc[q]);
    if (s == 3) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        finite = finite && isfinite(acc[q]);
        d[q] = d[q] - h6 * acc[q];
      }
      t.clamp_box(d);
    }
  }
  return finite;
}

// One node: particle creation (i), backward RK4 (ii), T evaluation (iii).
// The node is entry `tid` of chunk ck = (macro, slab p1, first index, count).
template <int D, class R, bool STEADY, int P = 2, int MODE = kStep, int BLEND = 0>
__device__ __forceinline__ void advect_node(const NodeJob<R>& job, Tables<R> tab, int4 ck, int tid) {
  const StepConsts<R>& K = job.K;
  const int npm = job.npm;
  constexpr int TIE_DF = (MODE != kStep && sizeof(R) == 4) ? 1 : 0;
  Tracer<D, R, STEADY, P, BLEND, TIE_DF> t;
  t.geo = job.geo;
  t.tab = tab;
  t.N = job.N;
  t.npm = npm;
  t.nmac = job.n_macros;
  t.un = job.un;
  t.uo = job.uo;
  t.T = job.T_old;
  t.dt = K.dt;
  t.Nf = K.Nf;
  t.invM = K.invM;
  t.status = job.status;
  t.load_block_macro(ck.x);
  // (i) particle creation at the node (an interface copy starts from its owner's lattice point)
  t.m0 = ck.x;
  const int i = ck.z + tid;  // index within slab p1
  t.p[0] = ck.y;
  int in_macro;
  if (D == 3) {
    const int p2 = tri_root2<D>(i);
    t.p[1] = p2;
    t.p[D - 1] = i - tri2(p2);
    in_macro = tri3(ck.y) + i;
  } else {
    t.p[D - 1] = i;
    in_macro = tri2(ck.y) + i;
  }
  const int64_t slot = int64_t(t.m0) * npm + in_macro;
  {
    const int M = P * job.N;
    bool iface = t.p[0] == M || t.p[D - 1] == 0;
#pragma unroll
    for (int k = 1; k < D; ++k) iface = iface || t.p[k] == t.p[k - 1];
    if (iface) {
      const int64_t own = job.owner_mp[job.unique_map[slot]];
      t.m0 = unpack_owner<D>(own, t.p);
      // one owner per node (Sec. 2.3.1): a copy held by another macro is
      // filled from its owner's slot after the step
      if (job.skip_ghosts && t.m0 != ck.x) return;
    }
  }
  {
#pragma unroll
    for (int q = 0; q < D; ++q) {
      R x = tab.v0(t.m0, q);
#pragma unroll
      for (int c = 0; c < D; ++c) x = r_fma(tab.J(t.m0, q * 3 + c), to_real<R>(t.p[c]) * K.invM, x);
      t.dlo[q] = K.lo[q] - x;
      t.dhi[q] = K.hi[q] - x;
      if constexpr (BLEND == 1) t.xc[q] = double(x);
    }
    if constexpr (BLEND == 1) {
      t.bl = job.bl;
      blend_fwd(job.bl, t.xc[0], t.xc[1], t.xp);
    }
  }
  t.home_frame();
  const int own_slot = t.m0 * npm + packed<D>(t.p);
  R d[D];
  bool from_node = true;
#pragma unroll
  for (int q = 0; q < D; ++q) d[q] = R(0);
  if (MODE != kStep && job.D_in != nullptr) {
    // every copy of an interface node continues from its owner's offset
#pragma unroll
    for (int q = 0; q < D; ++q) d[q] = job.D_in[int64_t(own_slot) * D + q];
    t.clamp_box(d);
    from_node = false;
  }
  bool finite = true;
  if (MODE != kEval) {
    R u_node[D];
    Tracer<D, R, STEADY, P, BLEND, TIE_DF>::load_rec(t.un, own_slot, u_node);
    finite = rk4_backward<D>(t, K, job.n_sub, u_node, from_node, d);
  }
  if (MODE == kTrace) {
    if (!finite) atomicOr(job.status, kFlagNonFinite);
#pragma unroll
    for (int q = 0; q < D; ++q) job.D_out[slot * D + q] = d[q];
    return;
  }
  // (iii) temperature at the departure point
  const R v = t.scalar(d);
  finite = finite && isfinite(v);
  if (!finite) atomicOr(job.status, kFlagNonFinite);
  job.T_new[slot] = v;
}


}  // namespace
}  // namespace elm
