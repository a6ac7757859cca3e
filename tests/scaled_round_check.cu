// scaled_round_check.cu -- CPU check of elm::scaled_round (the adjoint's
// FP32-to-integer conversion): for finite FP32 c and every scale k with
// |c 2^k| < 2^61 (the range the adjoint's slot scales allow) it must give the
// integer llrint(ldexp(double(c), k)) computes, ties to even included.
// Cases: random magnitudes over the whole FP32 range, exact halves and
// quarter steps (ties), subnormals, the largest and the smallest scales.
// Built with nvcc (host code) and run by tests/test_scaled_round.py.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "scaled_round.cuh"

int main() {
  std::mt19937_64 g(11);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  long long n = 0, bad = 0;
  for (int it = 0; it < 4000000; ++it) {
    float c;
    const int kind = it % 4;
    if (kind == 0) {
      c = float(std::ldexp(u(g), int(g() % 250) - 125));  // normal range
    } else if (kind == 1) {
      c = float(std::ldexp(double(int(g() % 129) - 64), -int(g() % 4)));  // ties at k = 0
    } else if (kind == 2) {
      const unsigned b = unsigned(g()) & 0x807fffffu;  // subnormal (or zero)
      std::memcpy(&c, &b, sizeof c);
    } else {
      const unsigned b = unsigned(g()) & 0xff7fffffu;  // any finite bit pattern
      std::memcpy(&c, &b, sizeof c);
    }
    if (c == 0.0f || !std::isfinite(c)) continue;
    int e;
    std::frexp(double(c), &e);  // |c| < 2^e
    const int kmax = 61 - e;    // |c 2^kmax| < 2^61
    const int ks[4] = {kmax, kmax - int(g() % 40), kmax - int(g() % 90), 0};
    for (int j = 0; j < 4; ++j) {
      const int k = ks[j];
      if (k > kmax) continue;
      const long long want = std::llrint(std::ldexp(double(c), k));
      const long long got = elm::scaled_round(c, k);
      ++n;
      if (got != want) {
        if (bad < 10) std::printf("mismatch: c = %a, k = %d: %lld, want %lld\n", double(c), k, got, want);
        ++bad;
      }
    }
  }
  std::printf("%lld cases, %lld mismatches\n", n, bad);
  if (bad == 0) std::printf("all ok\n");
  return bad != 0;
}
