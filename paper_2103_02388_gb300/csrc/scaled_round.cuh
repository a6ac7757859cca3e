// scaled_round.cuh -- round(c 2^k) to the nearest 64-bit integer, ties to
// even, for an FP32 c, by integer shifts of its significand.
//
// The adjoint adds each contribution c to a slot as the integer
// round(c 2^k_slot) (deterministic sums, see adjoint.cu).  Written in
// floating point that is llrint(ldexp(double(c), k)): three FP64 operations
// per contribution, which run on GB300's narrow FP64 pipe.  Here
// c = m 2^(e - 150) with the 24-bit integer significand m (e the biased
// exponent, 1 for subnormals), so c 2^k = m 2^s with s = e - 150 + k: a left
// shift for s >= 0, otherwise a right shift by -s rounded to nearest even
// from the bits shifted out.  The result is the same integer for every finite
// c with |c 2^k| < 2^62 (the slot scales keep |c 2^k| < 2^61), and needs no
// floating-point operation.  Host and device: a CPU test (nvcc host code)
// checks it against llrint(ldexp()).
#pragma once

#include <cstdint>
#include <cstring>

namespace elm {

__host__ __device__ __forceinline__ unsigned scaled_round_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

__host__ __device__ __forceinline__ long long scaled_round(float c, int k) {
  const unsigned b = scaled_round_bits(c);
  const int e = int((b >> 23) & 0xffu);
  const unsigned long long m = (b & 0x7fffffu) | (e != 0 ? 0x800000u : 0u);
  const int s = (e != 0 ? e : 1) - 150 + k;
  unsigned long long r;
  if (s >= 0) {
    r = s < 64 ? m << s : 0ull;
  } else if (s < -25) {
    r = 0ull;  // m 2^s < 2^(24 + s) <= 2^-2
  } else {
    const int t = -s;  // 1 .. 25
    const unsigned long long q = m >> t, rem = m & ((1ull << t) - 1ull), half = 1ull << (t - 1);
    r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  return (b >> 31) ? -(long long)r : (long long)r;
}

}  // namespace elm
