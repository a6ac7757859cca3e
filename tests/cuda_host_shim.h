// cuda_host_shim.h -- host stand-ins for the CUDA device built-ins and
// intrinsics that the kernels' device code uses, so that the same source
// compiles with g++ and runs on the CPU (under AddressSanitizer /
// UndefinedBehaviorSanitizer) in the host check programs of tests/.
//
// Each stand-in states the operation's meaning in plain C++: bit casts by
// memcpy, conversions with the rounding the intrinsic's name gives (rn: to
// nearest even, rd: down, rz: toward zero; out-of-range values saturate),
// fused multiply-adds by std::fma, and atomics as plain read-modify-writes when
// the host program runs one thread at a time.  CUDA_HOST_THREADS switches to
// running each block's threads together (barriers, warp exchanges, atomic
// built-ins; end of this file).  Test infrastructure only.
#pragma once

#include <cuda_runtime.h>  // vector types (float2, int4, ...), dim3, uint3

#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstdint>
#include <cstring>

// The launch geometry.  Without CUDA_HOST_THREADS the host program runs one
// GPU thread at a time (kernels without barriers or warp exchanges); with it,
// host_launch below runs each block's threads as host threads together.
#ifdef CUDA_HOST_THREADS
inline thread_local uint3 threadIdx, blockIdx;
#else
inline uint3 threadIdx, blockIdx;
#endif
inline dim3 blockDim, gridDim;

// qualifiers nvcc knows and a host compiler does not
#undef __noinline__
#define __noinline__
#define __launch_bounds__(...)
#define __grid_constant__
#define __shared__ static  // blocks run one after another, so one copy serves each block
#ifndef CUDA_HOST_THREADS
inline void __syncthreads() {}
#endif

using std::frexp;
using std::isfinite;
using std::isnan;
using std::ldexp;
using std::llrint;
using std::signbit;

// bit casts
inline unsigned __float_as_uint(float x) { unsigned u; std::memcpy(&u, &x, 4); return u; }
inline float __uint_as_float(unsigned u) { float x; std::memcpy(&x, &u, 4); return x; }
inline int __float_as_int(float x) { int u; std::memcpy(&u, &x, 4); return u; }
inline float __int_as_float(int u) { float x; std::memcpy(&x, &u, 4); return x; }
inline long long __double_as_longlong(double x) { long long u; std::memcpy(&u, &x, 8); return u; }
inline double __longlong_as_double(long long u) { double x; std::memcpy(&x, &u, 8); return x; }
inline int __double2hiint(double x) { return int(__double_as_longlong(x) >> 32); }
inline int __double2loint(double x) { return int(__double_as_longlong(x) & 0xffffffffLL); }
inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((unsigned long long)(unsigned)hi << 32) | (unsigned)lo));
}

// conversions (saturating, NaN to INT_MIN)
inline int shim_saturate(long double v) {
  if (std::isnan(double(v))) return INT_MIN;
  if (v >= 2147483647.0L) return INT_MAX;
  if (v <= -2147483648.0L) return INT_MIN;
  return int(v);
}
inline int __float2int_rn(float x) { return shim_saturate(std::nearbyint((long double)x)); }
inline int __float2int_rd(float x) { return shim_saturate(std::floor((long double)x)); }
inline int __float2int_rz(float x) { return shim_saturate(std::trunc((long double)x)); }
inline int __double2int_rn(double x) { return shim_saturate(std::nearbyint((long double)x)); }
inline int __double2int_rd(double x) { return shim_saturate(std::floor((long double)x)); }
inline int __double2int_rz(double x) { return shim_saturate(std::trunc((long double)x)); }
inline float __int2float_rn(int i) { return float(i); }
inline double __int2double_rn(int i) { return double(i); }
inline float __ll2float_rn(long long v) { return float(v); }

// arithmetic with a stated rounding
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
}
inline float2 __fmul2_rn(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
inline float2 __fadd2_rn(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline int max(int a, int b) { return a > b ? a : b; }
inline int min(int a, int b) { return a < b ? a : b; }
inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
inline unsigned min(unsigned a, unsigned b) { return a < b ? a : b; }
inline long long max(long long a, long long b) { return a > b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline unsigned long long max(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
inline unsigned long long min(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
inline float max(float a, float b) { return std::fmax(a, b); }
inline float min(float a, float b) { return std::fmin(a, b); }
inline double max(double a, double b) { return std::fmax(a, b); }
inline double min(double a, double b) { return std::fmin(a, b); }

// loads and bit counts
template <class T>
inline T __ldg(const T* p) { return *p; }
inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
inline int __ffs(int x) { return __builtin_ffs(x); }

// atomics (one thread at a time)
inline unsigned atomicOr(unsigned* p, unsigned v) { unsigned o = *p; *p |= v; return o; }
inline unsigned atomicAdd(unsigned* p, unsigned v) { unsigned o = *p; *p += v; return o; }
inline int atomicAdd(int* p, int v) { int o = *p; *p += v; return o; }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  unsigned long long o = *p;
  *p += v;
  return o;
}
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
  unsigned long long o = *p;
  if (v > o) *p = v;
  return o;
}

#ifndef CUDA_HOST_THREADS
// kernel() runs once per thread of a grid of `blocks` blocks of `threads`
// threads, one thread at a time (kernels without barriers or warp exchanges).
template <class F>
void host_serial_launch(unsigned blocks, unsigned threads, F kernel) {
  gridDim = dim3(blocks, 1, 1);
  blockDim = dim3(threads, 1, 1);
  for (unsigned b = 0; b < blocks; ++b) {
    blockIdx = make_uint3(b, 0, 0);
    for (unsigned t = 0; t < threads; ++t) {
      threadIdx = make_uint3(t, 0, 0);
      kernel();
    }
  }
}
#endif

#ifdef CUDA_HOST_THREADS
// Blocks run one after another; the threads of a block run together as host
// threads.  __syncthreads is a barrier over the block's threads that have not
// returned; a warp exchange (the shuffles) is a barrier over the warp's 32
// threads, which all take part (full masks), with the values passed through
// a per-warp table.  Atomics are the compiler's atomic built-ins.
#include <array>
#include <atomic>
#include <barrier>
#include <memory>
#include <thread>
#include <vector>

struct HostBlock {
  std::unique_ptr<std::barrier<>> block;
  std::vector<std::unique_ptr<std::barrier<>>> warp;
  std::vector<std::array<unsigned long long, 32>> xchg;
};
inline HostBlock* g_host_block = nullptr;

inline void __syncthreads() { g_host_block->block->arrive_and_wait(); }
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
template <class T>
inline T __ldcg(const T* p) {
  T v;
  __atomic_load(p, &v, __ATOMIC_SEQ_CST);
  return v;
}

template <class T>
inline T host_warp_exchange(T v, unsigned src) {
  static_assert(sizeof(T) <= 8, "one 64-bit word per lane");
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  unsigned long long bits = 0;
  std::memcpy(&bits, &v, sizeof(T));
  g_host_block->xchg[w][lane] = bits;
  g_host_block->warp[w]->arrive_and_wait();
  const unsigned long long r = g_host_block->xchg[w][src];
  g_host_block->warp[w]->arrive_and_wait();
  T out;
  std::memcpy(&out, &r, sizeof(T));
  return out;
}
template <class T>
inline T __shfl_down_sync(unsigned, T v, unsigned o) {
  const unsigned lane = threadIdx.x & 31u;
  return host_warp_exchange(v, lane + o < 32u ? lane + o : lane);  // out of range: the lane's own value
}
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int m) {
  return host_warp_exchange(v, (threadIdx.x & 31u) ^ unsigned(m));
}

// kernel() runs once per thread of a grid of `blocks` blocks of `threads`
// threads (a multiple of 32).
template <class F>
void host_launch(unsigned blocks, unsigned threads, F kernel) {
  if (threads == 0 || threads % 32 != 0) std::abort();  // whole warps only
  gridDim = dim3(blocks, 1, 1);
  blockDim = dim3(threads, 1, 1);
  for (unsigned b = 0; b < blocks; ++b) {
    HostBlock hb;
    hb.block = std::make_unique<std::barrier<>>(std::ptrdiff_t(threads));
    for (unsigned w = 0; w < threads / 32; ++w) hb.warp.push_back(std::make_unique<std::barrier<>>(32));
    hb.xchg.resize(threads / 32);
    g_host_block = &hb;
    std::vector<std::thread> th;
    th.reserve(threads);
    for (unsigned t = 0; t < threads; ++t)
      th.emplace_back([&, t] {
        threadIdx = make_uint3(t, 0, 0);
        blockIdx = make_uint3(b, 0, 0);
        kernel();
        // a returned thread is no longer waited for, by the block or its warp
        // (a lane that returns before a warp exchange its warp still makes
        // leaves that exchange's value undefined, as on the GPU; the results
        // then differ instead of the emulation hanging)
        hb.block->arrive_and_drop();
        hb.warp[t / 32]->arrive_and_drop();
      });
    for (auto& x : th) x.join();
    g_host_block = nullptr;
  }
}

#define atomicAdd(p, v) host_atomic_add_any(p, v)
template <class T, class V>
inline T host_atomic_add_any(T* p, V v) { return __atomic_fetch_add(p, T(v), __ATOMIC_SEQ_CST); }
#endif
