// adjoint_kernels.cuh -- device code of the adjoint of the advection step:
// the per-node reverse sweep (k_adjoint, one kernel per pass) and the
// per-slot kernels around it (statistics of interface copies, scale
// exponents, folding of the copies' sums, scaling back).  The method, the
// deterministic fixed-point sums and the launch sequence are described in
// adjoint.cu, which includes this file; kept apart from the launches so
// that the device code also compiles as host code for the CPU checks.
#pragma once

#include <cstdint>

#include "scaled_round.cuh"
#include "tracer.cuh"

namespace elm {
namespace {

constexpr int kSumBits = 61;   // |sum of a slot| < 2^61 (64-bit accumulators)

struct AdjArgs {
  const void* gT_new;
  unsigned long long* acc_T;   // [n] int64
  unsigned long long* acc_U;   // [nsets][dim][n] int64 (component-major)
  // per slot statistics and scales: T slots [0, n), velocity slots
  // [n + set n, n + (set + 1) n)
  unsigned long long* smax;    // largest |contribution| (value bits)
  unsigned long long* scnt;    // number of contributions
  const int* kexp;             // scale exponent k_j
  int split;                   // u_old and u_new gradients kept apart
  int pass;                    // 0: statistics, 1: accumulate (selects the kernel)
};

template <class R>
struct Bits;
template <>
struct Bits<float> {
  static __device__ unsigned long long of(float x) { return (unsigned long long)__float_as_uint(fabsf(x)); }
  static __device__ float from(unsigned long long b) { return __uint_as_float(unsigned(b)); }
};
template <>
struct Bits<double> {
  static __device__ unsigned long long of(double x) { return (unsigned long long)__double_as_longlong(::fabs(x)); }
  static __device__ double from(unsigned long long b) { return __longlong_as_double((long long)b); }
};

// Scale exponent of a slot whose contributions number cnt with largest
// magnitude m: cnt m 2^k < 2^kSumBits (m < 2^e, cnt <= 2^b).  e from frexpf
// for an FP32 m (the same exponent as of its exact double, without the FP64
// pipe), from frexp for an FP64 one.
template <class R>
__device__ __forceinline__ int scale_exponent(R m, unsigned long long cnt) {
  if (cnt == 0ull || !(m > R(0)) || !isfinite(m)) return 0;
  int e;
  if constexpr (sizeof(R) == 4)
    frexpf(m, &e);  // m < 2^e
  else
    frexp(m, &e);
  const int b = cnt <= 1ull ? 0 : 64 - __clzll((long long)(cnt - 1ull));
  return kSumBits - b - e;
}

// PASS 0 gathers the slot statistics, PASS 1 the scaled sums: a kernel per
// pass, so that each carries only its own accumulation code.
template <int D, class R, bool STEADY, int P, int PASS>
struct Adjoint {
  using Tr = Tracer<D, R, STEADY, P>;
  static constexpr int NB = Tr::NB;
  Tr t;
  AdjArgs A;
  int n_storage;
  R h, h2, h6;
  int n_sub;
  int home_slot;

  __device__ void clamp_mask(R* z, unsigned& mask) const {
    mask = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const R v = r_clamp(z[k], t.dlo[k], t.dhi[k]);
      if (v != z[k]) mask |= 1u << k;
      z[k] = v;
    }
  }

  // round(c 2^k) as a 64-bit integer: by integer shifts in FP32 (no FP64
  // conversion; the same integer, scaled_round.cuh), llrint in FP64.
  static __device__ __forceinline__ long long to_fixed(R c, int k) {
    if constexpr (sizeof(R) == 4)
      return scaled_round(c, k);
    else
      return llrint(ldexp(c, k));
  }

  // Contribution c to dL/dT^n at slot: its statistics (pass 0) or its scaled
  // integer (pass 1).  Zero contributions are skipped in both passes.
  __device__ void addT(int slot, R c) {
    if (c == R(0)) return;
    if constexpr (PASS == 0) {
      atomicMax(A.smax + slot, Bits<R>::of(c));
      atomicAdd(A.scnt + slot, 1ull);
      return;
    }
    const long long q = to_fixed(c, A.kexp[slot]);
    atomicAdd(A.acc_T + slot, (unsigned long long)q);
  }
  // Contribution v[0..D) to the velocity gradient of set `set` at slot: one
  // statistic (the largest component; the integer order of the value bits
  // puts NaN above every number) and one scale for the slot's components.
  __device__ void addU(int set, int slot, const R* v) {
    const int64_t st = int64_t(n_storage) * (1 + set) + slot;
    if constexpr (PASS == 0) {
      unsigned long long mb = 0ull;
#pragma unroll
      for (int r = 0; r < D; ++r) mb = max(mb, Bits<R>::of(v[r]));
      if (mb == 0ull) return;
      atomicMax(A.smax + st, mb);
      atomicAdd(A.scnt + st, 1ull);
      return;
    }
    const int k = A.kexp[st];
#pragma unroll
    for (int r = 0; r < D; ++r)
      if (v[r] != R(0))
        atomicAdd(A.acc_U + (int64_t(set) * D + r) * n_storage + slot,
                  (unsigned long long)to_fixed(v[r], k));
  }

  // P1 / P2 stencil with barycentrics L and the axis of each sorted fraction.
  __device__ void stencil_ad(const R* c, const R* f, int* slot, R* phi, R* L, int* ax) const {
    t.stencil(c, f, slot, phi);
    // recompute the sorted order (same comparisons as stencil)
    R fs[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      fs[k] = f[k];
      ax[k] = k;
    }
    auto cswap = [&](int i, int j) {
      if (r_greater(fs[j], fs[i])) {
        R tmp = fs[i]; fs[i] = fs[j]; fs[j] = tmp;
        int u = ax[i]; ax[i] = ax[j]; ax[j] = u;
      }
    };
    if (D == 3) { cswap(0, 1); cswap(1, 2); cswap(0, 1); } else { cswap(0, 1); }
    L[0] = R(1) - fs[0];
#pragma unroll
    for (int v = 1; v < D; ++v) L[v] = fs[v - 1] - fs[v];
    L[D] = fs[D - 1];
  }

  // Physical gradient of a P1 / P2 field with stencil values hv at the
  // located point (barycentrics L, sorted axes ax), in the current macro
  // frame.  G_v is the derivative with respect to barycentric L_v: the vertex
  // value for P1 (the basis is L itself, in the stencil's vertex order), the
  // derivative of the vertex and edge terms for P2.
  __device__ void grad_x(const R* hv, const R* L, const int* ax, R* gx) const {
    R G[D + 1];
    if constexpr (P == 1) {
#pragma unroll
      for (int v = 0; v <= D; ++v) G[v] = hv[v];
    } else if (D == 3) {
      G[0] = hv[0] * (R(4) * L[0] - R(1)) + R(4) * (L[1] * hv[4] + L[2] * hv[5] + L[D] * hv[6]);
      G[1] = hv[1] * (R(4) * L[1] - R(1)) + R(4) * (L[0] * hv[4] + L[2] * hv[7] + L[D] * hv[8]);
      G[2] = hv[2] * (R(4) * L[2] - R(1)) + R(4) * (L[0] * hv[5] + L[1] * hv[7] + L[D] * hv[9 % NB]);
      G[D] = hv[3] * (R(4) * L[D] - R(1)) + R(4) * (L[0] * hv[6] + L[1] * hv[8] + L[2] * hv[9 % NB]);
    } else {
      G[0] = hv[0] * (R(4) * L[0] - R(1)) + R(4) * (L[1] * hv[3] + L[D] * hv[4]);
      G[1] = hv[1] * (R(4) * L[1] - R(1)) + R(4) * (L[0] * hv[3] + L[D] * hv[5]);
      G[D] = hv[2] * (R(4) * L[D] - R(1)) + R(4) * (L[0] * hv[4] + L[1] * hv[5]);
    }
    // d/d fs_k = G_{k+1} - G_k; fs_k is the fraction along axis ax[k]
    R gq[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      R v = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) v = ax[k] == a ? G[k + 1] - G[k] : v;
      gq[a] = v;
    }
    // q = NJinv (x - v0): grad_x = NJinv^T grad_q
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
      R v = R(0);
#pragma unroll
      for (int r = 0; r < D; ++r) v = r_fma(t.nj(r * D + cc), gq[r], v);
      gx[cc] = v;
    }
  }

  // Forward substeps j0 .. j1-1 from offset d (no trace kept).
  __device__ void forward(R* d, int j0, int j1) {
    for (int j = j0; j < j1; ++j) {
      const R back = to_real<R>(j) * h;
      R k[D], acc[D], z[D];
      if (j == 0) {
        R un[D];
        Tr::load_rec(t.un, home_slot, un);
#pragma unroll
        for (int q = 0; q < D; ++q) k[q] = un[q];
      } else {
        t.velocity(d, back, k);
      }
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = k[q];
#pragma unroll 1
      for (int s = 1; s < 4; ++s) {
        const R off = s == 3 ? h : h2;
#pragma unroll
        for (int q = 0; q < D; ++q) z[q] = d[q] - off * k[q];
        t.clamp_box(z);
        t.velocity(z, back + off, k);
        const R w = s == 3 ? R(1) : R(2);
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = r_fma(w, k[q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < D; ++q) d[q] = d[q] - h6 * acc[q];
      t.clamp_box(d);
    }
  }

  // Reverse of one velocity evaluation k = u~(z) at backward time `back`:
  // scatters phi_j a_k to the velocity gradient and returns J_u(z)^T a_k.
  __device__ void velocity_adjoint(const R* z, R back, const R* ak, R* az) {
    R c[D], f[D];
    t.locate(z, c, f);
    int slot[NB];
    R phi[NB], L[D + 1];
    int ax[D];
    stencil_ad(c, f, slot, phi, L, ax);
    R w_old = R(0), w_new = R(1);
    if constexpr (!STEADY) {
      w_old = back / t.dt;
      w_new = (t.dt - back) / t.dt;
    }
    R hv[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      R un[D];
      Tr::load_rec(t.un, slot[j], un);
      R v = R(0);
#pragma unroll
      for (int r = 0; r < D; ++r) v = r_fma(ak[r], un[r], v);
      if constexpr (!STEADY) {
        R uo[D];
        Tr::load_rec(t.uo, slot[j], uo);
        R vo = R(0);
#pragma unroll
        for (int r = 0; r < D; ++r) vo = r_fma(ak[r], uo[r], vo);
        v = w_new * v + w_old * vo;
      }
      hv[j] = v;
    }
    grad_x(hv, L, ax, az);
    auto scatter = [&](int sl, R ph) {
      R pa[D];
#pragma unroll
      for (int r = 0; r < D; ++r) pa[r] = ph * ak[r];
      if (STEADY || !A.split) {
        addU(0, sl, pa);
      } else {
        R po[D], pn[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
          po[r] = w_old * pa[r];
          pn[r] = w_new * pa[r];
        }
        addU(0, sl, po);
        addU(1, sl, pn);
      }
    };
    // The scatter of the summing pass (conversions and atomics for every
    // component) and every FP64 scatter run as a loop, for code size; the
    // FP32 statistics pass keeps it unrolled (measured faster).
    if constexpr (PASS == 1 || sizeof(R) == 8) {
#pragma unroll 1
      for (int j = 0; j < NB; ++j) scatter(slot[j], phi[j]);
    } else {
#pragma unroll
      for (int j = 0; j < NB; ++j) scatter(slot[j], phi[j]);
    }
  }

  // Stage points z_s of one substep and the coordinates its clamps fixed
  // (mz[s] for z_s, md for the end point).
  struct Stages {
    R z[4][D];
    unsigned mz[4], md;
  };

  // Forward substep j from offset d, keeping its stage points and clamps; d
  // becomes the substep's end point (the same arithmetic as forward()).
  // The stage loop is not unrolled: one inlined copy of the velocity
  // evaluation instead of four keeps the kernel's code small enough for the
  // instruction cache (instruction fetch was the largest stall of the
  // unrolled form); the stage arrays go to the stack frame.
  // Keep a single call site: with two inlined copies of this rolled loop in
  // run() the compiled kernels (nvcc 13.0, sm_103a; ptxas at -O0 as at its
  // default level, and with FMA contraction off) computed wrong velocity
  // gradients, although the two source forms are equivalent (a host build of
  // both gives bitwise the same sums); with one copy, or the first copy
  // unrolled, they pass every parity test.
  __device__ void substep(R* d, int j, Stages& st) {
    const R back = to_real<R>(j) * h;
    R k[4][D], acc[D];
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      const R off = s == 3 ? h : h2;
      R zs[D], ks[D];
      unsigned m = 0u;
      if (s == 0) {
#pragma unroll
        for (int q = 0; q < D; ++q) zs[q] = d[q];
      } else {
#pragma unroll
        for (int q = 0; q < D; ++q) zs[q] = d[q] - off * k[s - 1][q];
        clamp_mask(zs, m);
      }
      if (s == 0 && j == 0)
        Tr::load_rec(t.un, home_slot, ks);
      else
        t.velocity(zs, s == 0 ? back : back + off, ks);
#pragma unroll
      for (int q = 0; q < D; ++q) {
        st.z[s][q] = zs[q];
        k[s][q] = ks[q];
      }
      st.mz[s] = m;
    }
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = k[0][q];
#pragma unroll
    for (int s = 1; s < 4; ++s) {
      const R w = s == 3 ? R(1) : R(2);
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = r_fma(w, k[s][q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < D; ++q) d[q] = d[q] - h6 * acc[q];
    clamp_mask(d, st.md);
  }

  __device__ void run(R g) {
    // forward to the start of the last substep; the reverse loop below runs
    // each substep's stages once (the last one also gives the departure point)
    R X[D];
#pragma unroll
    for (int q = 0; q < D; ++q) X[q] = R(0);
    forward(X, 0, n_sub - 1);
    Stages st;
    R a[D];
    // (ii) reverse through the substeps, last first; substep jj < n_sub - 1
    // is replayed from the start node, and the last one is run only here
    // (not also in the forward pass above)
    for (int jj = n_sub - 1; jj >= 0; --jj) {
      R d[D];
      if (jj == n_sub - 1) {
#pragma unroll
        for (int q = 0; q < D; ++q) d[q] = X[q];
      } else {
#pragma unroll
        for (int q = 0; q < D; ++q) d[q] = R(0);
        forward(d, 0, jj);
      }
      substep(d, jj, st);
      if (jj == n_sub - 1) {
        // (iii) T^{n+1} = T_h(X): transpose interpolation and a_X = g grad T_h(X)
        R c[D], f[D];
        t.locate(d, c, f);
        int slot[NB];
        R phi[NB], L[D + 1];
        int ax[D];
        stencil_ad(c, f, slot, phi, L, ax);
        R hv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          hv[j] = __ldg(t.T + slot[j]);
          addT(slot[j], phi[j] * g);
        }
        grad_x(hv, L, ax, a);
#pragma unroll
        for (int q = 0; q < D; ++q) a[q] *= g;
      }
      const R back = to_real<R>(jj) * h;
      // reverse: d_end = clamp(d - h/6 (k0 + 2 k1 + 2 k2 + k3))
      R ak[4][D], ad[D];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const R ap = (st.md >> q) & 1u ? R(0) : a[q];
        ad[q] = ap;
        ak[0][q] = -h6 * ap;
        ak[1][q] = R(-2) * h6 * ap;
        ak[2][q] = R(-2) * h6 * ap;
        ak[3][q] = -h6 * ap;
      }
#pragma unroll 1
      for (int s = 3; s >= 0; --s) {
        R as[D];
#pragma unroll
        for (int q = 0; q < D; ++q) as[q] = ak[s][q];
        if (s == 0 && jj == 0) {
          // first stage: the nodal value of u^{n+1} (weight 1 at t_{n+1})
          addU(STEADY || !A.split ? 0 : 1, home_slot, as);
          break;
        }
        const R off = s == 3 ? h : h2;
        R zs[D], az[D];
#pragma unroll
        for (int q = 0; q < D; ++q) zs[q] = st.z[s][q];
        velocity_adjoint(zs, s == 0 ? back : back + off, as, az);
        if (s > 0) {
#pragma unroll
          for (int q = 0; q < D; ++q) {
            const R v = (st.mz[s] >> q) & 1u ? R(0) : az[q];
            ad[q] += v;                 // z_s = d - off k_{s-1}
            ak[s - 1][q] -= off * v;
          }
        } else {
#pragma unroll
          for (int q = 0; q < D; ++q) ad[q] += az[q];
        }
      }
#pragma unroll
      for (int q = 0; q < D; ++q) a[q] = ad[q];
    }
  }
};

template <int D, class R, bool STEADY, int P, int PASS>
__global__ void __launch_bounds__(kAdvectThreads)
    k_adjoint(AdvectArgs args, AdjArgs aa, Tables<R> tab, int chunk0) {
  const int4 ck = args.chunks[chunk0 + int(blockIdx.x)];
  if (int(threadIdx.x) >= ck.w) return;
  const StepConsts<R>& K = consts<R>(args);
  const int npm = int(args.npm);
  Adjoint<D, R, STEADY, P, PASS> ad;
  Tracer<D, R, STEADY, P>& t = ad.t;
  t.geo = args.geo;
  t.tab = tab;
  t.N = args.N;
  t.npm = npm;
  t.un = static_cast<const R*>(args.u_new);
  t.uo = static_cast<const R*>(args.u_old);
  t.T = static_cast<const R*>(args.T_old);
  t.dt = K.dt;
  t.Nf = K.Nf;
  t.invM = K.invM;
  t.status = args.status;
  t.load_block_macro(ck.x);
  ad.A = aa;
  ad.n_storage = int(args.n_storage);
  ad.h = K.h;
  ad.h2 = K.h2;
  ad.h6 = K.h6;
  ad.n_sub = args.n_sub;
  // node and owner, as in the forward step
  t.m0 = ck.x;
  const int i = ck.z + int(threadIdx.x);
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
  const int slot = t.m0 * npm + in_macro;
  const R g = static_cast<const R*>(aa.gT_new)[slot];
  if (g == R(0)) return;
  {
    const int M = P * args.N;
    bool iface = t.p[0] == M || t.p[D - 1] == 0;
#pragma unroll
    for (int k = 1; k < D; ++k) iface = iface || t.p[k] == t.p[k - 1];
    if (iface) {
      const int64_t own = args.owner_mp[args.unique_map[slot]];
      t.m0 = unpack_owner<D>(own, t.p);
    }
  }
#pragma unroll
  for (int q = 0; q < D; ++q) {
    R x = tab.v0(t.m0, q);
#pragma unroll
    for (int c = 0; c < D; ++c) x = r_fma(tab.J(t.m0, q * 3 + c), to_real<R>(t.p[c]) * K.invM, x);
    t.dlo[q] = K.lo[q] - x;
    t.dhi[q] = K.hi[q] - x;
  }
  t.home_frame();
  ad.home_slot = t.m0 * npm + packed<D>(t.p);
  ad.run(g);
}

// Interface copies: a copy's statistics are merged into its owner's (pass 0
// result), then the owner's scale is handed back to the copy, so both sum at
// one scale.  g = (copy slot, owner slot) pairs; one thread per (pair, set).
__global__ void k_merge_stats(unsigned long long* smax, unsigned long long* scnt, int64_t n, int nsets,
                              const int2* __restrict__ g, int n_ghosts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(n_ghosts) * nsets) return;
  const int set = int(i / n_ghosts);
  const int2 p = g[i - int64_t(set) * n_ghosts];
  const int64_t a = set * n + p.x, o = set * n + p.y;
  if (scnt[a] == 0ull) return;
  atomicMax(smax + o, smax[a]);
  atomicAdd(scnt + o, scnt[a]);
}
__global__ void k_copy_scales(int* kexp, int64_t n, int nsets, const int2* __restrict__ g, int n_ghosts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(n_ghosts) * nsets) return;
  const int set = int(i / n_ghosts);
  const int2 p = g[i - int64_t(set) * n_ghosts];
  kexp[set * n + p.x] = kexp[set * n + p.y];
}

// Scale exponents of every slot from its statistics; a non-finite largest
// contribution sets the status flag.
template <class R>
__global__ void k_scales(const unsigned long long* __restrict__ smax, const unsigned long long* __restrict__ scnt,
                         int* kexp, int64_t count, unsigned* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const R m = Bits<R>::from(smax[i]);
  if (scnt[i] != 0ull && !isfinite(m)) atomicOr(status, kFlagNonFinite);
  kexp[i] = scale_exponent<R>(m, scnt[i]);
}

// Ghost copies of a node hand their sums to the owner slot.
__global__ void k_fold_ghosts(unsigned long long* acc, int ncomp, int nsets, int64_t n,
                              const int64_t* __restrict__ unique_map, const int64_t* __restrict__ owner) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t o = owner[unique_map[s]];
  if (o == s) return;
  for (int set = 0; set < nsets; ++set)
    for (int c = 0; c < ncomp; ++c) {
      unsigned long long* src = acc + (int64_t(set) * ncomp + c) * n + s;
      const unsigned long long v = *src;
      if (v) {
        atomicAdd(acc + (int64_t(set) * ncomp + c) * n + o, v);
        *src = 0ull;
      }
    }
}

// out[s ncomp + c] = acc[c n + s] 2^-k_s: component-major sums back to the
// caller's interleaved layout (ncomp = 1 for the temperature), k_s the
// slot's scale exponent (shared by its components).  FP32: one correctly
// rounded conversion of the 64-bit sum, then an exact scaling (no FP64
// pipe); FP64: the same in double.
template <class R>
__global__ void k_scale_out(const unsigned long long* __restrict__ acc, R* __restrict__ out, int64_t n,
                            int ncomp, const int* __restrict__ kexp) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * ncomp) return;
  const int64_t sl = i / ncomp;
  const int c = int(i - sl * ncomp);
  const long long v = (long long)acc[c * n + sl];
  if constexpr (sizeof(R) == 4)
    out[i] = ldexpf(__ll2float_rn(v), -kexp[sl]);
  else
    out[i] = ldexp(double(v), -kexp[sl]);
}

}  // namespace
}  // namespace elm
