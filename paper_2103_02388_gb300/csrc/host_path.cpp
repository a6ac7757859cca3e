// host_path.cpp -- the advection step with host buffers (elm_advect_host):
// device staging in two alternating sets, copies on the mesh's own streams,
// and the step launched in pieces whose results go back while the rest is
// computed.  The step itself is the kernel of elm_advect (Algorithm 1,
// lines 3-4); this file only moves data and orders streams.
#include <algorithm>
#include <cmath>
#include <string>

#include "elm_internal.h"

namespace {

elm_status fail(elm_status s, const std::string& msg) {
  elm::set_last_error(msg);
  return s;
}

elm_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ELM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// True when the byte range [p, p + bytes) starts and ends in page-locked host
// memory known to CUDA.
bool page_locked(const void* p, size_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (const char* q : {c, c + (bytes > 0 ? bytes - 1 : 0)}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();  // clear the error state left by the failed query
      return false;
    }
    if (at.type != cudaMemoryTypeHost) return false;
  }
  return true;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return na > 0 && nb > 0 && pa < pb + nb && pb < pa + na;
}

// Storage slot of the first node of a work-list chunk (macro, p1, i0, count):
// slab p1 starts at the packed index of (p1, 0[, 0]).
int64_t chunk_first_slot(const elm_mesh_s* me, const int4& c) {
  const int64_t p1 = c.y;
  const int64_t slab = me->dim == 3 ? p1 * (p1 + 1) * (p1 + 2) / 6 : p1 * (p1 + 1) / 2;
  return int64_t(c.x) * me->npm + slab + c.z;
}

}  // namespace

namespace elm {

elm_status setup_host_staging(elm_mesh_s* me, std::string* err) {
  auto* H = new HostStaging();
  me->staging = H;
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  const size_t n = size_t(me->n_storage);
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (bytes == 0) return true;
    return cudaMalloc(p, bytes) == cudaSuccess;
  };
  bool ok = true;
  for (int k = 0; k < 2 && ok; ++k) {
    ok = alloc(&H->u[k][0], es * n * me->dim) && alloc(&H->u[k][1], es * n * me->dim) &&
         alloc(&H->T_old[k], es * n) && alloc(&H->T_new[k], es * n);
  }
  ok = ok && cudaStreamCreateWithFlags(&H->h2d, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&H->d2h, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) {
    ok = cudaEventCreateWithFlags(&H->ev_h2d[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&H->ev_d2h[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&H->ev_free[k], cudaEventDisableTiming) == cudaSuccess;
    for (int p = 0; p < kHostParts && ok; ++p)
      ok = cudaEventCreateWithFlags(&H->ev_part[k][p], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    *err = "out of device memory for the host staging buffers";
    return ELM_ERR_CUDA;
  }
  // pieces: near-equal runs of the work list; the chunks are in storage
  // order, so each run covers a contiguous storage range
  const int64_t nc = me->n_chunks;
  for (int p = 0; p <= kHostParts; ++p) {
    H->part_chunk[p] = nc * p / kHostParts;
    H->part_slot[p] = H->part_chunk[p] < nc ? chunk_first_slot(me, me->chunks[size_t(H->part_chunk[p])])
                                            : me->n_storage;
    // the piece's interface copies; their owners lie in this or an earlier
    // piece (an owner's slot precedes its copies')
    H->part_ghost[p] = std::lower_bound(me->ghosts.begin(), me->ghosts.end(), H->part_slot[p],
                                        [](const int2& g, int64_t v) { return g.x < v; }) -
                       me->ghosts.begin();
  }
  return ELM_OK;
}

void free_host_staging(elm_mesh_s* me) {
  HostStaging* H = me->staging;
  if (!H) return;
  if (H->h2d) cudaStreamSynchronize(H->h2d);
  if (H->d2h) cudaStreamSynchronize(H->d2h);
  for (int k = 0; k < 2; ++k) {
    cudaFree(H->u[k][0]);
    cudaFree(H->u[k][1]);
    cudaFree(H->T_old[k]);
    cudaFree(H->T_new[k]);
    for (cudaEvent_t e : {H->ev_h2d[k], H->ev_d2h[k], H->ev_free[k]})
      if (e) cudaEventDestroy(e);
    for (int p = 0; p < kHostParts; ++p)
      if (H->ev_part[k][p]) cudaEventDestroy(H->ev_part[k][p]);
  }
  if (H->h2d) cudaStreamDestroy(H->h2d);
  if (H->d2h) cudaStreamDestroy(H->d2h);
  delete H;
  me->staging = nullptr;
}

}  // namespace elm

extern "C" elm_status elm_advect_host(elm_mesh me, const void* u_old_host, const void* u_new_host,
                                      const void* T_old_host, void* T_new_host, double dt, int n_sub, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_advect_host: null mesh");
  // both velocity pointers null: the mesh's current velocity stays resident
  const bool keep_u = !u_old_host && !u_new_host;
  if ((!keep_u && (!u_old_host || !u_new_host)) || !T_old_host || !T_new_host)
    return fail(ELM_ERR_ARG, "elm_advect_host: null buffer");
  if (!std::isfinite(dt) || dt < 0.0) return fail(ELM_ERR_ARG, "elm_advect_host: dt must be finite and >= 0");
  if (n_sub < 1 || n_sub > elm::kMaxSub)
    return fail(ELM_ERR_ARG, "elm_advect_host: n_sub must be in 1.." + std::to_string(elm::kMaxSub));
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_advect_host: host-only mesh");
  if (!me->staging) return fail(ELM_ERR_STATE, "elm_advect_host: mesh was created without ELM_HOST_STAGING");
  if (keep_u && !me->have_velocity)
    return fail(ELM_ERR_STATE, "elm_advect_host: no velocity pointers and no velocity set on the mesh");
  const size_t es = me->precision == ELM_FP64 ? 8 : 4;
  const size_t tb = es * size_t(me->n_storage), ub = keep_u ? 0 : tb * size_t(me->dim);
  const bool steady = keep_u ? me->steady : u_old_host == u_new_host;
  DeviceGuard g(me->device);
  if ((!keep_u && (!page_locked(u_new_host, ub) || (!steady && !page_locked(u_old_host, ub)))) ||
      !page_locked(T_old_host, tb) || !page_locked(T_new_host, tb))
    return fail(ELM_ERR_ARG, "elm_advect_host: host buffers must be page-locked (cudaHostAlloc, cudaHostRegister)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "elm_advect_host");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(ELM_ERR_STATE, "elm_advect_host: not capturable (orders itself after the previous call)");

  elm::HostStaging& H = *me->staging;
  const int k = H.next, o = 1 - k;
  // 1. inputs to the device, on the copy stream: after the last use of set k,
  //    and after the host result in flight on set o if an input aliases it
  e = cudaStreamWaitEvent(H.h2d, H.ev_free[k], 0);
  if (e == cudaSuccess && H.out_bytes[o] > 0 &&
      (overlap(u_new_host, ub, H.out_ptr[o], H.out_bytes[o]) ||
       overlap(u_old_host, ub, H.out_ptr[o], H.out_bytes[o]) ||
       overlap(T_old_host, tb, H.out_ptr[o], H.out_bytes[o])))
    e = cudaStreamWaitEvent(H.h2d, H.ev_d2h[o], 0);
  if (e == cudaSuccess && !keep_u) e = cudaMemcpyAsync(H.u[k][1], u_new_host, ub, cudaMemcpyHostToDevice, H.h2d);
  if (e == cudaSuccess && !keep_u && !steady)
    e = cudaMemcpyAsync(H.u[k][0], u_old_host, ub, cudaMemcpyHostToDevice, H.h2d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(H.T_old[k], T_old_host, tb, cudaMemcpyHostToDevice, H.h2d);
  if (e == cudaSuccess) e = cudaEventRecord(H.ev_h2d[k], H.h2d);
  // 2. the velocity and the step on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, H.ev_h2d[k], 0);
  if (e == cudaSuccess && !keep_u)
    e = elm::launch_pack_velocity(me->precision, me->dim, H.u[k][1], me->d_u4[1], me->n_storage, s);
  if (e == cudaSuccess && !keep_u && !steady)
    e = elm::launch_pack_velocity(me->precision, me->dim, H.u[k][0], me->d_u4[0], me->n_storage, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_advect_host");
  me->steady = steady;
  me->have_velocity = true;
  elm::AdvectArgs a = elm::make_args(me, dt, n_sub);
  a.T_old = H.T_old[k];
  a.T_new = H.T_new[k];
  // 3. piece by piece: the step on `stream`, its result back on the other
  //    copy stream as soon as the piece is done
  char* out = static_cast<char*>(T_new_host);
  const char* dev_out = static_cast<const char*>(H.T_new[k]);
  for (int p = 0; p < elm::kHostParts && e == cudaSuccess; ++p) {
    const int64_t c0 = H.part_chunk[p], c1 = H.part_chunk[p + 1];
    const int64_t s0 = H.part_slot[p], s1 = H.part_slot[p + 1];
    if (c1 > c0) {
      a.chunks = me->d_chunks + c0;
      a.n_chunks = int(c1 - c0);
      a.ghosts = me->d_ghosts + H.part_ghost[p];
      a.n_ghosts = int(H.part_ghost[p + 1] - H.part_ghost[p]);
      e = elm::launch_advect(me->dim, me->precision, a, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(H.ev_part[k][p], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(H.d2h, H.ev_part[k][p], 0);
    if (e == cudaSuccess && s1 > s0)
      e = cudaMemcpyAsync(out + size_t(s0) * es, dev_out + size_t(s0) * es, size_t(s1 - s0) * es,
                          cudaMemcpyDeviceToHost, H.d2h);
  }
  // 4. the caller's stream completes after the result is on the host; the
  //    set is free again from there
  if (e == cudaSuccess) e = cudaEventRecord(H.ev_d2h[k], H.d2h);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, H.ev_d2h[k], 0);
  if (e == cudaSuccess) e = cudaEventRecord(H.ev_free[k], s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_advect_host");
  H.out_ptr[k] = out;
  H.out_bytes[k] = tb;
  H.next = o;
  return ELM_OK;
}
