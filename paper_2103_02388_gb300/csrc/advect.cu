// advect.cu -- the MMOC advection step on sm_103a (arXiv 2103.02388, Sec. 2.3.1
// steps (i)-(iii), Eq. departure point, Eq. linear interpolation,
// Algorithm 1 lines 3-4).
//
// One thread per storage node.  A thread creates its particle at node x_i
// (step (i)), traces it backwards with n_sub classic RK4 substeps through the
// P2 velocity (step (ii)) and interpolates T^n at the departure point
// (step (iii)).  All macros are resident in HBM, so the paper's particle
// migration between processes becomes an in-register macro walk.  A node on
// a macro interface is stored once per macro holding it and is computed once,
// by the thread of its owner copy (the single-owner rule of Sec. 2.3.1, grid
// data structure); the threads of the other copies return at once, and
// k_ghost_copy then copies the owner's value into them, so all copies hold
// bitwise the same value.  The batched kernel does the same, with one copy
// pass for all its instances.
//
// Point representation.  A point is kept as an offset d from its start node
// x_i, and its level-L lattice coordinate in the current macro m as
// q = b + r0 + NJinv_m d with an integer-valued part b and a small fraction
// r0 of the start node.  b carries the node's absolute position exactly, so
// FP32 keeps full precision in the fractional coordinates that decide the
// micro element, independent of the macro's size.  When the walk enters
// another macro, (b, r0) of the start node are recomputed in that macro's
// frame: in FP64 for the FP64 kernel, in double-float arithmetic on the FP32
// pipe for the FP32 kernel.
//
// Field evaluation (Sec. 2.3.2, field evaluation):
//   macro   -- barycentrics l = (N - q1, q1 - q2, q2 - q3, q3) in lattice
//              units; if min l < -tol the walk hops across the face opposite
//              the most negative one (at most kMaxHops hops);
//   micro   -- cell c = floor(q), fractions f = q - c; the Kuhn simplex of
//              the cell is given by the descending order of f (O(1));
//   P2 sum  -- micro barycentrics L = (1 - f_s0, f_s0 - f_s1, f_s1 - f_s2,
//              f_s2); vertex basis L(2L - 1), edge basis 4 L_a L_b.
// In FP32, a hop decision across an interior macro face whose barycentric
// lies within kBand32 of 0 is re-taken in FP64 from the exact start node.
//
// GB300 notes.  FP64 runs at a small fraction of the FP32 rate on this part,
// so the FP32 kernel keeps every FP64 (and double-float) instruction in
// non-inlined rare-path functions (the compiler would otherwise hoist the
// loop-invariant FP64 start-node position into every thread).  Lattice
// integers are integer-valued floats.  Every block works inside one macro,
// so that macro's N J^{-1} is held once per thread as a block-uniform value
// and a foreign macro's is read from the L1-resident table after a hand-off.  The packed index of a lattice point is separable,
// idx(p) = T3(p1) + T2(p2) + p3, so the 10 P2 nodes of a micro simplex are
// sums of three per-axis table entries; the tables are sorted together with
// the fractions, which leaves 2 integer adds per node.
#include <cstdint>

#include "tracer.cuh"

namespace elm {
namespace {

// kAdvectSplit blocks per work-list chunk: a chunk is a run of up to
// kAdvectThreads consecutive nodes of one slab p1 of one macro (host-built, so
// no thread divides or searches for its lattice point beyond one row root),
// and block b takes the nodes [(b mod kAdvectSplit) kStepThreads, ...) of
// chunk b / kAdvectSplit.
// P is the element order (1 or 2), MODE what is done per node (NodeMode),
// BLEND whether the mesh is blended onto an annulus.
template <int D, class R, bool STEADY, int P, int MODE, int BLEND>
__global__ void __launch_bounds__(kStepThreads, ELM_ADVECT_MIN_BLOCKS * kAdvectSplit)
    k_advect(AdvectArgs args, Tables<R> tab, int chunk0) {
  const int4 ck = args.chunks[chunk0 + int(blockIdx.x) / kAdvectSplit];
  const int tid = (int(blockIdx.x) % kAdvectSplit) * kStepThreads + int(threadIdx.x);
  if (tid >= ck.w) return;
  NodeJob<R> job{args.geo,
                       static_cast<const R*>(args.u_new),
                       static_cast<const R*>(args.u_old),
                       static_cast<const R*>(args.T_old),
                       static_cast<R*>(args.T_new),
                       args.status,
                       args.unique_map,
                       args.owner_mp,
                       consts<R>(args),
                       args.N,
                       int(args.npm),
                       args.n_sub,
                       static_cast<const R*>(args.D_in),
                       static_cast<R*>(args.D_out)};
  if constexpr (BLEND == 1) {
    job.bl = args.blend;
    job.n_macros = args.n_macros;
  }
  job.skip_ghosts = args.skip_ghosts;
  advect_node<D, R, STEADY, P, MODE, BLEND>(job, tab, ck, tid);
}

// Persistent batched kernel: each block repeatedly takes the next work item
// (instance, run of consecutive chunks) from the work list and advects those
// chunks' nodes with the instance's tables and this call's constants.
// Dimension and steadiness are per instance and uniform within a block; the
// element order P is per launch (a batch that mixes P1 and P2 instances runs
// one launch per order over its own part of the work list).  MINB is the
// number of resident blocks per SM the register budget is sized for.  As in
// k_advect, each interface node is computed once, by its owner copy; the
// copies are filled by k_batch_ghost_copy afterwards.
template <class R>
__device__ __forceinline__ Tables<R> tables_of(const BatchStatic& S);
template <>
__device__ __forceinline__ Tables<float> tables_of<float>(const BatchStatic& S) { return Tables<float>{S.geo32}; }
template <>
__device__ __forceinline__ Tables<double> tables_of<double>(const BatchStatic& S) { return Tables<double>{S.geo}; }

template <class R, int P, int MINB>
__global__ void __launch_bounds__(kAdvectThreads, MINB)
    k_advect_batch(const __grid_constant__ BatchParams<R> B) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(B.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= B.n_items) return;
    const int4 w = B.items[it];
    const BatchStatic& S = B.inst[w.x];
    const BatchCall<R>& C = B.call[w.x];
    for (int cc = 0; cc < w.z; ++cc) {
      const int4 ck = S.chunks[w.y + cc];
      if (int(threadIdx.x) < ck.w) {
        NodeJob<R> job{S.geo,
                       static_cast<const R*>(C.u_new),
                       static_cast<const R*>(C.u_old),
                       static_cast<const R*>(C.T_old),
                       static_cast<R*>(C.T_new),
                       S.status,
                       S.unique_map,
                       S.owner_mp,
                       C.K,
                       S.N,
                       S.npm,
                       C.n_sub};
        job.skip_ghosts = 1;
        const Tables<R> tab = tables_of<R>(S);
        const int tid = int(threadIdx.x);
        if (S.dim == 3) {
          if (C.steady) advect_node<3, R, true, P>(job, tab, ck, tid);
          else advect_node<3, R, false, P>(job, tab, ck, tid);
        } else {
          if (C.steady) advect_node<2, R, true, P>(job, tab, ck, tid);
          else advect_node<2, R, false, P>(job, tab, ck, tid);
        }
      }
    }
  }
}

// Interface copies of every instance of a batch (a5): T_new[g.y] = T_new[g.z]
// of instance g.x, for the (instance, copy slot, owner slot) triples g.
template <class R>
__global__ void k_batch_ghost_copy(const __grid_constant__ BatchParams<R> B, const int4* __restrict__ g, int n) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 t = g[i];
  R* out = static_cast<R*>(B.call[t.x].T_new);
  out[t.y] = out[t.z];
}

// [n, dim] -> packed records [n, 4] (x, y[, z], 0).
template <class R>
__global__ void k_pack_velocity(const R* __restrict__ u, R* __restrict__ u4, int64_t n, int dim) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R w[4] = {R(0), R(0), R(0), R(0)};
  for (int r = 0; r < dim; ++r) w[r] = u[i * dim + r];
  for (int r = 0; r < 4; ++r) u4[i * 4 + r] = w[r];
}

// Interface copies (a5): out[ghost] = out[owner] for every (ghost slot,
// owner slot) pair, ncomp values per slot.
template <class R>
__global__ void k_ghost_copy(const int2* __restrict__ g, int n, R* __restrict__ out, int ncomp) {
  const int i = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * ncomp) return;
  const int j = i / ncomp, c = i - j * ncomp;
  const int2 p = g[j];
  out[int64_t(p.x) * ncomp + c] = out[int64_t(p.y) * ncomp + c];
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

template <int D, class R, bool STEADY, int P, int MODE>
cudaError_t launch_k(const AdvectArgs& a, Tables<R> t, cudaStream_t s) {
  const bool blended = a.blend.nsec > 0;
  if constexpr (D == 2 && sizeof(R) == 8) {
    if (blended) {
      for (int c0 = 0; c0 < a.n_chunks; c0 += (1 << 29)) {
        const int nb = a.n_chunks - c0 < (1 << 29) ? a.n_chunks - c0 : (1 << 29);
        k_advect<D, R, STEADY, P, MODE, 1><<<nb * kAdvectSplit, kStepThreads, 0, s>>>(a, t, c0);
      }
      return cudaGetLastError();
    }
  }
  if (blended) return cudaErrorInvalidValue;  // blending is 2D FP64 only (checked by the API)
  for (int c0 = 0; c0 < a.n_chunks; c0 += (1 << 29)) {
    const int nb = a.n_chunks - c0 < (1 << 29) ? a.n_chunks - c0 : (1 << 29);
    k_advect<D, R, STEADY, P, MODE, 0><<<nb * kAdvectSplit, kStepThreads, 0, s>>>(a, t, c0);
  }
  return cudaGetLastError();
}

template <int D, class R, int P>
cudaError_t launch_drp(const AdvectArgs& a, Tables<R> t, cudaStream_t s) {
  if (a.mode == kEval) return launch_k<D, R, true, P, kEval>(a, t, s);  // no velocity is read
  if (a.mode == kTrace)
    return a.steady ? launch_k<D, R, true, P, kTrace>(a, t, s) : launch_k<D, R, false, P, kTrace>(a, t, s);
  return a.steady ? launch_k<D, R, true, P, kStep>(a, t, s) : launch_k<D, R, false, P, kStep>(a, t, s);
}

template <int D, class R>
cudaError_t launch_dr(const AdvectArgs& a, Tables<R> t, cudaStream_t s) {
  return a.order == 1 ? launch_drp<D, R, 1>(a, t, s) : launch_drp<D, R, 2>(a, t, s);
}

}  // namespace

cudaError_t launch_advect(int dim, int precision, const AdvectArgs& a, cudaStream_t s) {
  if (a.n_storage == 0) return cudaSuccess;
  cudaError_t e;
  if (precision == ELM_FP64) {
    Tables<double> t{a.geo};
    e = dim == 3 ? launch_dr<3, double>(a, t, s) : launch_dr<2, double>(a, t, s);
  } else {
    Tables<float> t{a.geo32};
    e = dim == 3 ? launch_dr<3, float>(a, t, s) : launch_dr<2, float>(a, t, s);
  }
  if (e != cudaSuccess || !a.skip_ghosts || a.n_ghosts == 0) return e;
  // the per-node kernel skipped the non-owner copies: fill them
  const int ncomp = a.mode == kTrace ? dim : 1;
  void* out = a.mode == kTrace ? a.D_out : a.T_new;
  const unsigned blocks = unsigned((int64_t(a.n_ghosts) * ncomp + 255) / 256);
  if (precision == ELM_FP64)
    k_ghost_copy<double><<<blocks, 256, 0, s>>>(a.ghosts, a.n_ghosts, static_cast<double*>(out), ncomp);
  else
    k_ghost_copy<float><<<blocks, 256, 0, s>>>(a.ghosts, a.n_ghosts, static_cast<float*>(out), ncomp);
  return cudaGetLastError();
}

cudaError_t launch_batch32(const BatchParams<float>& p, int order, int min_blocks, int grid, cudaStream_t s) {
  if (min_blocks >= 8) {
    if (order == 1) k_advect_batch<float, 1, 8><<<grid, kAdvectThreads, 0, s>>>(p);
    else k_advect_batch<float, 2, 8><<<grid, kAdvectThreads, 0, s>>>(p);
  } else {
    if (order == 1) k_advect_batch<float, 1, 6><<<grid, kAdvectThreads, 0, s>>>(p);
    else k_advect_batch<float, 2, 6><<<grid, kAdvectThreads, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch64(const BatchParams<double>& p, int order, int min_blocks, int grid, cudaStream_t s) {
  if (min_blocks >= 8) {
    if (order == 1) k_advect_batch<double, 1, 8><<<grid, kAdvectThreads, 0, s>>>(p);
    else k_advect_batch<double, 2, 8><<<grid, kAdvectThreads, 0, s>>>(p);
  } else {
    if (order == 1) k_advect_batch<double, 1, 6><<<grid, kAdvectThreads, 0, s>>>(p);
    else k_advect_batch<double, 2, 6><<<grid, kAdvectThreads, 0, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_ghosts32(const BatchParams<float>& p, const int4* g, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_batch_ghost_copy<float><<<unsigned((n + 255) / 256), 256, 0, s>>>(p, g, n);
  return cudaGetLastError();
}

cudaError_t launch_batch_ghosts64(const BatchParams<double>& p, const int4* g, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_batch_ghost_copy<double><<<unsigned((n + 255) / 256), 256, 0, s>>>(p, g, n);
  return cudaGetLastError();
}

cudaError_t launch_pack_velocity(int precision, int dim, const void* u, void* u4, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const unsigned blocks = unsigned((n + 255) / 256);
  if (precision == ELM_FP64)
    k_pack_velocity<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(u), static_cast<double*>(u4), n, dim);
  else
    k_pack_velocity<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(u), static_cast<float*>(u4), n, dim);
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
