// adjoint.cu -- the adjoint of the advection step (arXiv 2103.02388: Eq.
// departure point and step (iii) of Sec. 2.3.1, differentiated).
//
// For T^{n+1}_i = T^n_h(X_i(u)) and an incoming gradient g = dL/dT^{n+1}:
//   dL/dT^n_j  = sum_i phi_j(X_i) g_i                (transpose interpolation)
//   dL/du_j    = sum_i g_i grad T^n_h(X_i) . dX_i/du_j  (reverse mode through
//                the backward RK4 stages, the P1 / P2 velocity evaluations, the
//                time interpolation and the box clamps)
// Each node i recomputes its forward trace (a substep is replayed from the
// start for every substep it reverses, so no trace is stored), then runs
// reverse mode: a stage k_s = u~(z_s) sends phi_j(z_s) a_k to node j's
// velocity and J_u(z_s)^T a_k back to z_s, where J_u is the gradient of the
// P1 / P2 interpolant; a clamped coordinate passes no derivative.
//
// Deterministic scatter-add: every contribution c is accumulated as a 64-bit
// integer round(c * 2^k) with integer atomics, which add exactly and in any
// order to the same sum.  A first pass finds the largest |c| (atomic max of
// the value bits) and fixes k so that 2^10 contributions of that size still
// fit; a second pass accumulates; ghost copies are folded into their owner
// slot and the sums are scaled back.  No floating-point atomics.
#include <cstdint>

#include "tracer.cuh"

namespace elm {
namespace {

constexpr int kHeadroomBits = 10;   // up to 2^10 maximal contributions per node
constexpr int kAccBits = 62;

struct AdjArgs {
  const void* gT_new;
  unsigned long long* acc_T;   // [n] int64
  unsigned long long* acc_U;   // [nsets][n][dim] int64
  unsigned long long* maxbits; // [2]: |contribution| maxima (T, U) as value bits
  int split;                   // u_old and u_new gradients kept apart
  int pass;                    // 0: maxima, 1: accumulate
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

// 2^k scale from the largest contribution m (power of two: c * 2^k is exact).
__device__ __forceinline__ int scale_exponent(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 0;
  int e;
  frexp(m, &e);  // m < 2^e
  return kAccBits - kHeadroomBits - e;
}

template <int D, class R, bool STEADY, int P>
struct Adjoint {
  using Tr = Tracer<D, R, STEADY, P>;
  static constexpr int NB = Tr::NB;
  Tr t;
  AdjArgs A;
  int n_storage;
  double sT, sU;       // pass 1: scales 2^k
  R h, h2, h6;
  int n_sub;
  int home_slot;
  R maxT, maxU;        // pass 0: running maxima of this thread

  __device__ void clamp_mask(R* z, unsigned& mask) const {
    mask = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const R v = r_clamp(z[k], t.dlo[k], t.dhi[k]);
      if (v != z[k]) mask |= 1u << k;
      z[k] = v;
    }
  }

  // Adds contribution c to accumulator slot (pass 1) or tracks its size (pass 0).
  __device__ void addT(int slot, R c) {
    if (A.pass == 0) {
      maxT = fmax(maxT, R(fabs(c)));
      return;
    }
    const long long q = llrint(double(c) * sT);
    atomicAdd(A.acc_T + slot, (unsigned long long)q);
  }
  __device__ void addU(int set, int slot, int r, R c) {
    if (A.pass == 0) {
      maxU = fmax(maxU, R(fabs(c)));
      return;
    }
    const long long q = llrint(double(c) * sU);
    atomicAdd(A.acc_U + (int64_t(set) * n_storage + slot) * D + r, (unsigned long long)q);
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
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int r = 0; r < D; ++r) {
        const R pa = phi[j] * ak[r];
        if (STEADY || !A.split) {
          addU(0, slot[j], r, pa);
        } else {
          addU(0, slot[j], r, w_old * pa);
          addU(1, slot[j], r, w_new * pa);
        }
      }
  }

  __device__ void run(R g) {
    // forward to the departure point
    R X[D];
#pragma unroll
    for (int q = 0; q < D; ++q) X[q] = R(0);
    forward(X, 0, n_sub);
    // (iii) T^{n+1} = T_h(X): transpose interpolation and a_X = g grad T_h(X)
    R a[D];
    {
      R c[D], f[D];
      t.locate(X, c, f);
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
    // (ii) reverse through the substeps, last first
    for (int jj = n_sub - 1; jj >= 0; --jj) {
      R d[D];
#pragma unroll
      for (int q = 0; q < D; ++q) d[q] = R(0);
      forward(d, 0, jj);
      const R back = to_real<R>(jj) * h;
      // forward substep jj, keeping its stage points, values and clamps
      R z[4][D], k[4][D], acc[D];
      unsigned mz[4] = {0u, 0u, 0u, 0u}, md = 0u;
#pragma unroll
      for (int q = 0; q < D; ++q) z[0][q] = d[q];
      if (jj == 0) {
        R un[D];
        Tr::load_rec(t.un, home_slot, un);
#pragma unroll
        for (int q = 0; q < D; ++q) k[0][q] = un[q];
      } else {
        t.velocity(z[0], back, k[0]);
      }
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = k[0][q];
#pragma unroll
      for (int s = 1; s < 4; ++s) {
        const R off = s == 3 ? h : h2;
#pragma unroll
        for (int q = 0; q < D; ++q) z[s][q] = d[q] - off * k[s - 1][q];
        clamp_mask(z[s], mz[s]);
        t.velocity(z[s], back + off, k[s]);
        const R w = s == 3 ? R(1) : R(2);
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = r_fma(w, k[s][q], acc[q]);
      }
      {
        R dn[D];
#pragma unroll
        for (int q = 0; q < D; ++q) dn[q] = d[q] - h6 * acc[q];
        clamp_mask(dn, md);
      }
      // reverse: d_end = clamp(d - h/6 (k0 + 2 k1 + 2 k2 + k3))
      R ak[4][D], ad[D];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const R ap = (md >> q) & 1u ? R(0) : a[q];
        ad[q] = ap;
        ak[0][q] = -h6 * ap;
        ak[1][q] = R(-2) * h6 * ap;
        ak[2][q] = R(-2) * h6 * ap;
        ak[3][q] = -h6 * ap;
      }
#pragma unroll
      for (int s = 3; s >= 1; --s) {
        const R off = s == 3 ? h : h2;
        R az[D];
        velocity_adjoint(z[s], back + off, ak[s], az);
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const R v = (mz[s] >> q) & 1u ? R(0) : az[q];
          ad[q] += v;                 // z_s = d - off k_{s-1}
          ak[s - 1][q] -= off * v;
        }
      }
      if (jj == 0) {
        // first stage: the nodal value of u^{n+1} (weight 1 at t_{n+1})
#pragma unroll
        for (int r = 0; r < D; ++r) addU(STEADY || !A.split ? 0 : 1, home_slot, r, ak[0][r]);
      } else {
        R az[D];
        velocity_adjoint(z[0], back, ak[0], az);
#pragma unroll
        for (int q = 0; q < D; ++q) ad[q] += az[q];
      }
#pragma unroll
      for (int q = 0; q < D; ++q) a[q] = ad[q];
    }
  }
};

template <int D, class R, bool STEADY, int P>
__global__ void __launch_bounds__(kAdvectThreads)
    k_adjoint(AdvectArgs args, AdjArgs aa, Tables<R> tab, int chunk0) {
  const int4 ck = args.chunks[chunk0 + int(blockIdx.x)];
  if (int(threadIdx.x) >= ck.w) return;
  const StepConsts<R>& K = consts<R>(args);
  const int npm = int(args.npm);
  Adjoint<D, R, STEADY, P> ad;
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
  ad.maxT = R(0);
  ad.maxU = R(0);
  ad.sT = ad.sU = 0.0;
  if (aa.pass == 1) {
    ad.sT = ldexp(1.0, scale_exponent(double(Bits<R>::from(aa.maxbits[0]))));
    ad.sU = ldexp(1.0, scale_exponent(double(Bits<R>::from(aa.maxbits[1]))));
  }
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
  if (aa.pass == 0) {
    if (!isfinite(ad.maxT) || !isfinite(ad.maxU)) atomicOr(args.status, kFlagNonFinite);
    atomicMax(aa.maxbits + 0, Bits<R>::of(ad.maxT));
    atomicMax(aa.maxbits + 1, Bits<R>::of(ad.maxU));
  }
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
      unsigned long long* src = acc + (set * n + s) * ncomp + c;
      const unsigned long long v = *src;
      if (v) {
        atomicAdd(acc + (set * n + o) * ncomp + c, v);
        *src = 0ull;
      }
    }
}

// out = acc * 2^-k (k from the recorded maximum).
template <class R>
__global__ void k_scale_out(const unsigned long long* __restrict__ acc, R* __restrict__ out, int64_t count,
                            const unsigned long long* __restrict__ maxbits, int which) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int k = scale_exponent(double(Bits<R>::from(maxbits[which])));
  out[i] = R(double((long long)acc[i]) * ldexp(1.0, -k));
}

template <int D, class R, bool STEADY>
cudaError_t launch_adj_drs(const AdvectArgs& a, const AdjArgs& aa, Tables<R> t, cudaStream_t s) {
  if (a.order == 1)
    k_adjoint<D, R, STEADY, 1><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
  else
    k_adjoint<D, R, STEADY, 2><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
  return cudaGetLastError();
}

template <int D, class R>
cudaError_t launch_adj_dr(const AdvectArgs& a, const AdjArgs& aa, Tables<R> t, cudaStream_t s) {
  return a.steady ? launch_adj_drs<D, R, true>(a, aa, t, s) : launch_adj_drs<D, R, false>(a, aa, t, s);
}

}  // namespace

cudaError_t launch_adjoint(int dim, int precision, const AdvectArgs& a, const AdjointBuffers& b,
                           const void* gT_new, void* gT_old, void* gU_old, void* gU_new, cudaStream_t s) {
  const int64_t n = a.n_storage;
  const int nsets = (!a.steady && gU_new) ? 2 : 1;
  cudaError_t e = cudaMemsetAsync(b.acc_T, 0, sizeof(unsigned long long) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.acc_U, 0, sizeof(unsigned long long) * n * dim * nsets, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.maxbits, 0, sizeof(unsigned long long) * 2, s);
  if (e != cudaSuccess) return e;
  AdjArgs aa{gT_new, b.acc_T, b.acc_U, b.maxbits, nsets == 2 ? 1 : 0, 0};
  for (int pass = 0; pass < 2; ++pass) {
    aa.pass = pass;
    if (precision == ELM_FP64) {
      Tables<double> t{a.geo};
      e = dim == 3 ? launch_adj_dr<3, double>(a, aa, t, s) : launch_adj_dr<2, double>(a, aa, t, s);
    } else {
      Tables<float> t{a.geo32};
      e = dim == 3 ? launch_adj_dr<3, float>(a, aa, t, s) : launch_adj_dr<2, float>(a, aa, t, s);
    }
    if (e != cudaSuccess) return e;
  }
  const unsigned fb = unsigned((n + 255) / 256);
  k_fold_ghosts<<<fb, 256, 0, s>>>(b.acc_T, 1, 1, n, a.unique_map, b.owner);
  k_fold_ghosts<<<fb, 256, 0, s>>>(b.acc_U, dim, nsets, n, a.unique_map, b.owner);
  const unsigned tb = unsigned((n + 255) / 256);
  const unsigned ub = unsigned((n * dim + 255) / 256);
  if (precision == ELM_FP64) {
    k_scale_out<double><<<tb, 256, 0, s>>>(b.acc_T, static_cast<double*>(gT_old), n, b.maxbits, 0);
    k_scale_out<double><<<ub, 256, 0, s>>>(b.acc_U, static_cast<double*>(gU_old), n * dim, b.maxbits, 1);
    if (nsets == 2)
      k_scale_out<double><<<ub, 256, 0, s>>>(b.acc_U + n * dim, static_cast<double*>(gU_new), n * dim, b.maxbits, 1);
  } else {
    k_scale_out<float><<<tb, 256, 0, s>>>(b.acc_T, static_cast<float*>(gT_old), n, b.maxbits, 0);
    k_scale_out<float><<<ub, 256, 0, s>>>(b.acc_U, static_cast<float*>(gU_old), n * dim, b.maxbits, 1);
    if (nsets == 2)
      k_scale_out<float><<<ub, 256, 0, s>>>(b.acc_U + n * dim, static_cast<float*>(gU_new), n * dim, b.maxbits, 1);
  }
  return cudaGetLastError();
}

}  // namespace elm
