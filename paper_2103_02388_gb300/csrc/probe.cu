// probe.cu -- measured throughput of the SM pipes the advection kernels are
// bound by (a timed loop per instruction kind), for the compute side of the
// benchmark's roofline.  The paper has no counterpart: it only provides the
// peaks that a measured kernel time is compared with.
//
// Each probe kernel runs 8 independent dependency chains per thread (enough
// to cover the pipe latency with 8 warps per SM sub-partition) of one kind of
// instruction, over a grid of 8 resident 256-thread blocks per SM, and keeps
// its result alive through a conditional store (to a file-scope device
// variable) that depends on every chain.
#include <cstdint>
#include <string>

#include "elm_internal.h"

namespace elm {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

enum ProbeKind { kFfma = 0, kFfma2 = 1, kFminmax = 2, kIminmax = 3, kDfma = 4, kProbeKinds = 5 };

__device__ float g_probe_sink;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(int iters, float seed) {
  const float t = seed + 1e-3f * float(threadIdx.x);
  float a[kChains];
  float2 a2[kChains];
  int ia[kChains];
  double da[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    a[j] = t + float(j);
    a2[j] = make_float2(t + float(j), t - float(j));
    ia[j] = int(threadIdx.x) * 7 + j;
    da[j] = double(t) + double(j);
  }
  const double dm = double(0.999f - 1e-7f * seed), dc = double(1e-3f * seed);
  const float m = 0.999f - 1e-7f * seed, c = 1e-3f * seed;
  const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      // min / max: each step combines two chains' previous values (copied
      // first, so the 8 operations of a step are independent) and alternates
      // max and min, so no two steps fold
      float b[kChains];
      int ib[kChains];
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        b[j] = a[j];
        ib[j] = ia[j];
      }
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        if constexpr (KIND == kFfma) {
          a[j] = fmaf(a[j], m, c);
        } else if constexpr (KIND == kFfma2) {
          a2[j] = __ffma2_rn(a2[j], m2, c2);
        } else if constexpr (KIND == kDfma) {
          da[j] = fma(da[j], dm, dc);
        } else if constexpr (KIND == kFminmax) {
          a[j] = (r & 1) ? fmaxf(b[j], b[(j + 1) % kChains]) : fminf(b[j], b[(j + 3) % kChains]);
        } else {
          ia[j] = (r & 1) ? max(ib[j], ib[(j + 1) % kChains]) : min(ib[j], ib[(j + 3) % kChains]);
        }
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j] + a2[j].x + a2[j].y + float(ia[j]) + float(da[j]);
  if (s == 1234.5f) g_probe_sink = s;  // keeps the chains alive
}

template <int KIND>
cudaError_t run_probe(int grid, int iters, cudaStream_t s, float* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_probe<KIND><<<grid, kProbeThreads, 0, s>>>(2, 1.0f);  // warm-up
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    k_probe<KIND><<<grid, kProbeThreads, 0, s>>>(iters, 1.0f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace elm

extern "C" elm_status elm_probe_pipes(double* rates_host, int n, void* stream) {
  if (!rates_host || n < 5) {
    elm::set_last_error("elm_probe_pipes: need an output array of 5 doubles");
    return ELM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    elm::set_last_error(std::string("elm_probe_pipes: ") + cudaGetErrorString(e));
    return ELM_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = 8 * sms, iters = 4096;
  // operations per launch: threads x iterations x 8 steps x chains (x2 lanes for FFMA2)
  const double ops = double(grid) * elm::kProbeThreads * iters * 8 * elm::kChains;
  float ms[elm::kProbeKinds] = {0, 0, 0, 0, 0};
  e = elm::run_probe<elm::kFfma>(grid, iters, s, &ms[0]);
  if (e == cudaSuccess) e = elm::run_probe<elm::kFfma2>(grid, iters, s, &ms[1]);
  if (e == cudaSuccess) e = elm::run_probe<elm::kFminmax>(grid, iters, s, &ms[2]);
  if (e == cudaSuccess) e = elm::run_probe<elm::kIminmax>(grid, iters, s, &ms[3]);
  // FP64 FMAs: the FP64 pipe is narrow on this part, so fewer iterations
  if (e == cudaSuccess) e = elm::run_probe<elm::kDfma>(grid, iters / 16, s, &ms[4]);
  if (e != cudaSuccess) {
    elm::set_last_error(std::string("elm_probe_pipes: ") + cudaGetErrorString(e));
    return ELM_ERR_CUDA;
  }
  rates_host[0] = ops / (ms[0] * 1e-3);
  rates_host[1] = 2.0 * ops / (ms[1] * 1e-3);
  rates_host[2] = ops / (ms[2] * 1e-3);
  rates_host[3] = ops / (ms[3] * 1e-3);
  rates_host[4] = ops / 16 / (ms[4] * 1e-3);
  return ELM_OK;
}
