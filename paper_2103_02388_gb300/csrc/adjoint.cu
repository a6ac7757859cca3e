// adjoint.cu -- the adjoint of the advection step (arXiv 2103.02388: Eq.
// departure point and step (iii) of Sec. 2.3.1, differentiated).
//
// For T^{n+1}_i = T^n_h(X_i(u)) and an incoming gradient g = dL/dT^{n+1}:
//   dL/dT^n_j  = sum_i phi_j(X_i) g_i                (transpose interpolation)
//   dL/du_j    = sum_i g_i grad T^n_h(X_i) . dX_i/du_j  (reverse mode through
//                the backward RK4 stages, the P1 / P2 velocity evaluations, the
//                time interpolation and the box clamps)
// Each node i recomputes its forward trace (substep j is replayed from the
// start when it is reversed, so no trace is stored; the last substep is run
// once and gives both the departure point and its reverse stages), then runs
// reverse mode: a stage k_s = u~(z_s) sends phi_j(z_s) a_k to node j's
// velocity and J_u(z_s)^T a_k back to z_s, where J_u is the gradient of the
// P1 / P2 interpolant; a clamped coordinate passes no derivative.
//
// Deterministic scatter-add with a scale per output slot: every contribution
// c to slot j is accumulated as the 64-bit integer round(c 2^k_j) with integer
// atomics, which add exactly and in any order to the same sum.  A first pass
// records, per slot, the largest |c| (atomic maximum of its value bits) and
// the number of contributions (atomic add); the storage copies of an
// interface node take their owner's statistics.  k_j is then chosen so that
// count_j * max_j 2^k_j < 2^61: the sum cannot leave the 64-bit range however
// many contributions a slot receives (a convergent flow that clamps many
// departure points onto one boundary node included), and each slot keeps
// about 61 - log2(count_j) bits relative to its own largest contribution, so
// small gradient entries keep their relative precision next to large ones.
// A second pass accumulates; the copies' sums are folded into the owner
// (same scale, exact) and every slot is scaled back.  No floating-point
// atomics.
#include "adjoint_kernels.cuh"

namespace elm {
namespace {

template <int D, class R, bool STEADY>
cudaError_t launch_adj_drs(const AdvectArgs& a, const AdjArgs& aa, Tables<R> t, cudaStream_t s) {
  if (a.order == 1) {
    if (aa.pass == 0)
      k_adjoint<D, R, STEADY, 1, 0><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
    else
      k_adjoint<D, R, STEADY, 1, 1><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
  } else {
    if (aa.pass == 0)
      k_adjoint<D, R, STEADY, 2, 0><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
    else
      k_adjoint<D, R, STEADY, 2, 1><<<a.n_chunks, kAdvectThreads, 0, s>>>(a, aa, t, 0);
  }
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
  const int64_t nstat = n * (1 + nsets);
  cudaError_t e = cudaMemsetAsync(b.acc_T, 0, sizeof(unsigned long long) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.acc_U, 0, sizeof(unsigned long long) * n * dim * nsets, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.smax, 0, sizeof(unsigned long long) * nstat, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.scnt, 0, sizeof(unsigned long long) * nstat, s);
  if (e != cudaSuccess) return e;
  AdjArgs aa{gT_new, b.acc_T, b.acc_U, b.smax, b.scnt, b.kexp, nsets == 2 ? 1 : 0, 0};
  const unsigned gb = unsigned((int64_t(b.n_ghosts) * (1 + nsets) + 255) / 256);
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
    if (pass == 0) {
      // scales: copies' statistics into their owner, exponents, owner's
      // exponent back to the copies
      if (b.n_ghosts > 0)
        k_merge_stats<<<gb, 256, 0, s>>>(b.smax, b.scnt, n, 1 + nsets, b.ghosts, b.n_ghosts);
      const unsigned sb = unsigned((nstat + 255) / 256);
      if (precision == ELM_FP64)
        k_scales<double><<<sb, 256, 0, s>>>(b.smax, b.scnt, b.kexp, nstat, a.status);
      else
        k_scales<float><<<sb, 256, 0, s>>>(b.smax, b.scnt, b.kexp, nstat, a.status);
      if (b.n_ghosts > 0) k_copy_scales<<<gb, 256, 0, s>>>(b.kexp, n, 1 + nsets, b.ghosts, b.n_ghosts);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  const unsigned fb = unsigned((n + 255) / 256);
  k_fold_ghosts<<<fb, 256, 0, s>>>(b.acc_T, 1, 1, n, a.unique_map, b.owner);
  k_fold_ghosts<<<fb, 256, 0, s>>>(b.acc_U, dim, nsets, n, a.unique_map, b.owner);
  const unsigned tb = unsigned((n + 255) / 256);
  const unsigned ub = unsigned((n * dim + 255) / 256);
  if (precision == ELM_FP64) {
    k_scale_out<double><<<tb, 256, 0, s>>>(b.acc_T, static_cast<double*>(gT_old), n, 1, b.kexp);
    k_scale_out<double><<<ub, 256, 0, s>>>(b.acc_U, static_cast<double*>(gU_old), n, dim, b.kexp + n);
    if (nsets == 2)
      k_scale_out<double><<<ub, 256, 0, s>>>(b.acc_U + n * dim, static_cast<double*>(gU_new), n, dim,
                                             b.kexp + 2 * n);
  } else {
    k_scale_out<float><<<tb, 256, 0, s>>>(b.acc_T, static_cast<float*>(gT_old), n, 1, b.kexp);
    k_scale_out<float><<<ub, 256, 0, s>>>(b.acc_U, static_cast<float*>(gU_old), n, dim, b.kexp + n);
    if (nsets == 2)
      k_scale_out<float><<<ub, 256, 0, s>>>(b.acc_U + n * dim, static_cast<float*>(gU_new), n, dim,
                                            b.kexp + 2 * n);
  }
  return cudaGetLastError();
}

}  // namespace elm
