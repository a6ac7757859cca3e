// batch.cpp -- C ABI of the batched form: many independent advection
// instances (meshes of different dimension and level, each with its own
// velocity, dt and n_sub) advanced by one persistent kernel launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "elm_internal.h"

struct elm_batch_s {
  int count = 0;
  int precision = ELM_FP64;
  int device = 0;
  int grid = 0;
  int n_items = 0;
  int n_items_p2 = 0;    // the work list holds the P2 instances' items first, then the P1 ones
  int min_blocks = 6;    // register budget of the kernel: 6 or 8 resident blocks per SM
  int chunks_per_item = 1;
  int n_ghosts = 0;
  std::vector<elm_mesh> meshes;
  elm::BatchStatic* d_inst = nullptr;
  int4* d_items = nullptr;
  int4* d_ghosts = nullptr;  // (instance, copy slot, owner slot) of every interface copy
  int* d_counter = nullptr;
};

namespace {

elm_status bfail(elm_status s, const std::string& msg) {
  elm::set_last_error(msg);
  return s;
}

struct BatchDevice {
  int prev = -1;
  explicit BatchDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~BatchDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void free_batch(elm_batch_s* b) {
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_ghosts);
  cudaFree(b->d_counter);
  b->d_inst = nullptr;
  b->d_items = nullptr;
  b->d_ghosts = nullptr;
  b->d_counter = nullptr;
}

template <class R>
void fill_consts(elm::StepConsts<R>& K, const elm_mesh_s* me, double dt, int n_sub) {
  const double h = dt / n_sub;
  K.h = R(h);
  K.h2 = R(0.5 * h);
  K.h6 = R(h / 6.0);
  K.dt = R(dt);
  K.invM = R(1.0 / me->M);
  K.Nf = R(me->N);
  for (int r = 0; r < 3; ++r) {
    K.lo[r] = R(me->lo[r]);
    K.hi[r] = R(me->hi[r]);
  }
}

template <class R>
elm_status launch(elm_batch_s* b, const void* const* T_old, void* const* T_new, const double* dt, const int* n_sub,
                  cudaStream_t s) {
  // ~20 KB of per-call data travels as the kernel's parameter block.
  elm::BatchParams<R>* P = new (std::nothrow) elm::BatchParams<R>();
  if (!P) return bfail(ELM_ERR_ARG, "elm_batch_advect: out of host memory");
  P->inst = b->d_inst;
  P->count = b->count;
  for (int k = 0; k < b->count; ++k) {
    const elm_mesh_s* me = b->meshes[k];
    elm::BatchCall<R>& c = P->call[k];
    c.u_new = me->d_u4[1];
    c.u_old = me->steady ? me->d_u4[1] : me->d_u4[0];
    c.steady = me->steady ? 1 : 0;
    c.T_old = T_old[k];
    c.T_new = T_new[k];
    c.n_sub = n_sub[k];
    fill_consts(c.K, me, dt[k], n_sub[k]);
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int), s);
  // one persistent launch per element order present, each over its part of
  // the work list with its own counter
  const int part[2][2] = {{0, b->n_items_p2}, {b->n_items_p2, b->n_items}};
  for (int o = 0; o < 2 && e == cudaSuccess; ++o) {
    if (part[o][1] == part[o][0]) continue;
    P->items = b->d_items + part[o][0];
    P->n_items = part[o][1] - part[o][0];
    P->counter = b->d_counter + o;
    if constexpr (sizeof(R) == 4) e = elm::launch_batch32(*P, o == 0 ? 2 : 1, b->min_blocks, b->grid, s);
    else e = elm::launch_batch64(*P, o == 0 ? 2 : 1, b->min_blocks, b->grid, s);
  }
  // the interface copies of every instance, from their owners
  if (e == cudaSuccess) {
    if constexpr (sizeof(R) == 4) e = elm::launch_batch_ghosts32(*P, b->d_ghosts, b->n_ghosts, s);
    else e = elm::launch_batch_ghosts64(*P, b->d_ghosts, b->n_ghosts, s);
  }
  delete P;
  if (e != cudaSuccess) return bfail(ELM_ERR_CUDA, std::string("elm_batch_advect: ") + cudaGetErrorString(e));
  return ELM_OK;
}

}  // namespace

extern "C" {

elm_status elm_batch_create(const elm_mesh* meshes, int count, int blocks_per_sm, int chunks_per_item,
                            elm_batch* out) {
  if (!out || !meshes) return bfail(ELM_ERR_ARG, "elm_batch_create: null argument");
  if (count < 1 || count > elm::kMaxBatch)
    return bfail(ELM_ERR_ARG, "elm_batch_create: count must be in 1.." + std::to_string(elm::kMaxBatch));
  if (blocks_per_sm < 0 || blocks_per_sm > 32) return bfail(ELM_ERR_ARG, "elm_batch_create: blocks_per_sm in 0..32");
  if (chunks_per_item < 0 || chunks_per_item > 64)
    return bfail(ELM_ERR_ARG, "elm_batch_create: chunks_per_item in 0..64");
  for (int k = 0; k < count; ++k) {
    if (!meshes[k]) return bfail(ELM_ERR_ARG, "elm_batch_create: null mesh " + std::to_string(k));
    if (meshes[k]->host_only) return bfail(ELM_ERR_STATE, "elm_batch_create: host-only mesh " + std::to_string(k));
    if (meshes[k]->blend.nsec > 0)
      return bfail(ELM_ERR_ARG, "elm_batch_create: blended meshes are not batched (mesh " + std::to_string(k) + ")");
    if (meshes[k]->precision != meshes[0]->precision)
      return bfail(ELM_ERR_ARG, "elm_batch_create: all meshes must share one precision");
    if (meshes[k]->device != meshes[0]->device)
      return bfail(ELM_ERR_ARG, "elm_batch_create: all meshes must live on one device");
  }
  elm_batch_s* b = new (std::nothrow) elm_batch_s();
  if (!b) return bfail(ELM_ERR_ARG, "elm_batch_create: out of host memory");
  b->count = count;
  b->precision = meshes[0]->precision;
  b->device = meshes[0]->device;
  b->meshes.assign(meshes, meshes + count);
  BatchDevice guard(b->device);
  int n_sm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return bfail(ELM_ERR_CUDA, std::string("elm_batch_create: ") + cudaGetErrorString(e));
  }
  const int bps = blocks_per_sm > 0 ? blocks_per_sm : 6;
  b->grid = n_sm * bps;
  b->min_blocks = bps >= 8 ? 8 : 6;
  b->chunks_per_item = chunks_per_item > 0 ? chunks_per_item : 1;
  // Static per-instance table, the work list of runs of chunks_per_item
  // consecutive chunks of one instance, and the interface copies.
  std::vector<elm::BatchStatic> inst(count);
  std::vector<int4> items;
  std::vector<int4> ghosts;
  for (int k = 0; k < count; ++k) {
    const elm_mesh_s* me = meshes[k];
    inst[k] = elm::BatchStatic{me->d_geo, me->d_geo32, me->d_unique_map, me->d_owner_mp, me->d_chunks,
                               me->d_status, me->N, int(me->npm), me->dim, 0};
  }
  const int G = b->chunks_per_item;
  for (int order : {2, 1}) {
    for (int k = 0; k < count; ++k)
      if (meshes[k]->order == order)
        for (int64_t c = 0; c < meshes[k]->n_chunks; c += G)
          items.push_back(make_int4(k, int(c), int(std::min<int64_t>(G, meshes[k]->n_chunks - c)), 0));
    if (order == 2) b->n_items_p2 = int(items.size());
  }
  b->n_items = int(items.size());
  for (int k = 0; k < count; ++k)
    for (const int2& g : meshes[k]->ghosts) ghosts.push_back(make_int4(k, g.x, g.y, 0));
  b->n_ghosts = int(ghosts.size());
  e = cudaMalloc(&b->d_inst, sizeof(elm::BatchStatic) * count);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, inst.data(), sizeof(elm::BatchStatic) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int4) * items.size());
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ghosts.empty()) e = cudaMalloc(&b->d_ghosts, sizeof(int4) * ghosts.size());
  if (e == cudaSuccess && !ghosts.empty())
    e = cudaMemcpy(b->d_ghosts, ghosts.data(), sizeof(int4) * ghosts.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(int));
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return bfail(ELM_ERR_CUDA, std::string("elm_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return ELM_OK;
}

elm_status elm_batch_destroy(elm_batch b) {
  if (!b) return ELM_OK;
  {
    BatchDevice guard(b->device);
    free_batch(b);
  }
  delete b;
  return ELM_OK;
}

int64_t elm_batch_num_items(elm_batch b) { return b ? b->n_items : 0; }

elm_status elm_batch_advect(elm_batch b, const void* const* T_old, void* const* T_new, const double* dt,
                            const int* n_sub, void* stream) {
  if (!b) return bfail(ELM_ERR_ARG, "elm_batch_advect: null batch");
  if (!T_old || !T_new || !dt || !n_sub) return bfail(ELM_ERR_ARG, "elm_batch_advect: null argument array");
  for (int k = 0; k < b->count; ++k) {
    const elm_mesh_s* me = b->meshes[k];
    const std::string who = "elm_batch_advect: instance " + std::to_string(k) + ": ";
    if (!me->have_velocity) return bfail(ELM_ERR_STATE, who + "elm_set_velocity has not been called");
    if (!T_old[k] || !T_new[k]) return bfail(ELM_ERR_ARG, who + "null temperature buffer");
    if (!std::isfinite(dt[k]) || dt[k] < 0.0) return bfail(ELM_ERR_ARG, who + "dt must be finite and >= 0");
    if (n_sub[k] < 1 || n_sub[k] > elm::kMaxSub)
      return bfail(ELM_ERR_ARG, who + "n_sub must be in 1.." + std::to_string(elm::kMaxSub));
    const size_t bytes = size_t(me->n_storage) * (me->precision == ELM_FP64 ? 8 : 4);
    const char* a = static_cast<const char*>(T_old[k]);
    const char* c = static_cast<const char*>(T_new[k]);
    if (a < c + bytes && c < a + bytes) return bfail(ELM_ERR_ARG, who + "T_old and T_new overlap");
  }
  BatchDevice guard(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return b->precision == ELM_FP32 ? launch<float>(b, T_old, T_new, dt, n_sub, s)
                                  : launch<double>(b, T_old, T_new, dt, n_sub, s);
}

}  // extern "C"
