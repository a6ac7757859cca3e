// noalloc.cu -- elm_advect_noalloc: the advection step for callers that may
// not allocate device memory at the call site.
//
// elm_advect reads the velocity from records that elm_set_velocity packed
// into buffers the mesh allocated.  This entry point takes the caller's
// [n, dim] velocity directly and packs it into a fixed scratch array that is
// part of the library image (a file-scope __device__ array), so the call
// itself never allocates or frees device memory.  It serves code that cannot
// call cudaMalloc where it advects: for example a host application whose
// device memory is handed out by its own pool and that forbids further
// cudaMalloc calls, or a time-critical loop in which the implicit device
// synchronisation of cudaMalloc / cudaFree is not acceptable.  The paper has
// no counterpart; it only changes where the working copy of the velocity lives.
#include <cmath>
#include <mutex>
#include <string>

#include "elm_internal.h"

namespace {

// Largest mesh (storage nodes) the static scratch can serve.
constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 19;
// Two packed velocity record buffers (u^{n+1}, u^n) at the widest record
// (4 doubles): 2 * 2^19 * 32 B = 32 MiB, held by every GPU that loads the
// library until the process exits.
constexpr size_t kRecordBytesMax = 4 * sizeof(double);
constexpr size_t kScratchBytes = size_t(2) * size_t(kNoAllocMaxNodes) * kRecordBytesMax;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal, resolved once per
// device on the first call (with that device current) and kept for the life
// of the process: a device whose primary context is destroyed and recreated
// after that first call (cudaDeviceReset) is not supported.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

struct CurrentDevice {
  int prev = -1;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

elm_status noalloc_fail(elm_status s, const std::string& msg) {
  elm::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" elm_status elm_advect_noalloc(elm_mesh me, const void* u_old_dev, const void* u_new_dev,
                                         const void* T_old_dev, void* T_new_dev, double dt, int n_sub,
                                         void* stream) {
  if (!me) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: null mesh");
  if (me->host_only) return noalloc_fail(ELM_ERR_STATE, "elm_advect_noalloc: host-only mesh");
  if (!u_old_dev || !u_new_dev) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: null velocity");
  if (!T_old_dev || !T_new_dev) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: null temperature buffer");
  if (!std::isfinite(dt) || dt < 0.0) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: dt must be finite and >= 0");
  if (n_sub < 1 || n_sub > elm::kMaxSub)
    return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: n_sub must be in 1.." + std::to_string(elm::kMaxSub));
  if (me->n_storage > kNoAllocMaxNodes)
    return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: mesh has " + std::to_string(me->n_storage) +
                                         " storage nodes, more than the static scratch limit of " +
                                         std::to_string(kNoAllocMaxNodes));
  const size_t esz = me->precision == ELM_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = size_t(me->n_storage) * esz;
  {
    const char* a = static_cast<const char*>(T_old_dev);
    const char* b = static_cast<const char*>(T_new_dev);
    if (a < b + bytes && b < a + bytes) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: T_old and T_new overlap");
  }
  if (me->device < 0 || me->device >= kMaxDevices) return noalloc_fail(ELM_ERR_ARG, "elm_advect_noalloc: device ordinal");
  CurrentDevice guard(me->device);

  // Set-up, once per device with that device current: the device address of
  // the static scratch array (its host-side name is only a stand-in).
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[me->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(ELM_ERR_CUDA, std::string("elm_advect_noalloc: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
      g_scratch_addr[me->device] = p;
    }
    scratch = g_scratch_addr[me->device];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool steady = u_old_dev == u_new_dev;
  void* rec_new = scratch;
  void* rec_old = static_cast<unsigned char*>(scratch) + size_t(kNoAllocMaxNodes) * kRecordBytesMax;
  // Every record component (including the zero pad) is written here, so no
  // part of the shared scratch needs clearing between calls.
  cudaError_t e = elm::launch_pack_velocity(me->precision, me->dim, u_new_dev, rec_new, me->n_storage, s);
  if (e == cudaSuccess && !steady)
    e = elm::launch_pack_velocity(me->precision, me->dim, u_old_dev, rec_old, me->n_storage, s);
  if (e != cudaSuccess) return noalloc_fail(ELM_ERR_CUDA, std::string("elm_advect_noalloc: ") + cudaGetErrorString(e));

  // Everything as elm_advect sets it (tables, step constants, the interface
  // copy pass), with the velocity records in the scratch array and the
  // caller's T buffers.
  elm::AdvectArgs a = elm::make_args(me, dt, n_sub);
  a.u_old = steady ? rec_new : rec_old;
  a.u_new = rec_new;
  a.steady = steady;
  a.T_old = T_old_dev;
  a.T_new = T_new_dev;
  e = elm::launch_advect(me->dim, me->precision, a, s);
  if (e != cudaSuccess) return noalloc_fail(ELM_ERR_CUDA, std::string("elm_advect_noalloc: ") + cudaGetErrorString(e));
  return ELM_OK;
}
