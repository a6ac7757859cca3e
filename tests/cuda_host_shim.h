// cuda_host_shim.h -- host stand-ins for the CUDA device built-ins and
// intrinsics that the advection kernels' device code (csrc/tracer.cuh) uses,
// so that the same source compiles with g++ and runs on the CPU (under
// AddressSanitizer / UndefinedBehaviorSanitizer) in tests/kernel_host_check.cpp.
//
// Each stand-in states the operation's meaning in plain C++: bit casts by
// memcpy, conversions with the rounding the intrinsic's name gives (rn: to
// nearest even, rd: down, rz: toward zero; out-of-range values saturate),
// fused multiply-adds by std::fma, and atomics as plain read-modify-writes (the
// host program runs one thread at a time).  Test infrastructure only.
#pragma once

#include <cuda_runtime.h>  // vector types (float2, int4, ...), dim3, uint3

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>

// the launch geometry of the block being emulated
inline uint3 threadIdx, blockIdx;
inline dim3 blockDim, gridDim;

// qualifiers nvcc knows and a host compiler does not
#undef __noinline__
#define __noinline__
#define __launch_bounds__(...)
#define __grid_constant__
#define __shared__ static
inline void __syncthreads() {}

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
