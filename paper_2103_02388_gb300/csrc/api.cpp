// api.cpp -- the C ABI of libelm.so (declared in include/elm.h).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <utility>

#include "elm_internal.h"

namespace {

thread_local std::string g_last_error;

elm_status fail(elm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

elm_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ELM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Makes the mesh's device current for the duration of a call.
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

size_t elem_size(const elm_mesh_s* me) { return me->precision == ELM_FP64 ? 8 : 4; }

void free_tables(elm_mesh_s* me) {
  elm::free_host_staging(me);
  cudaFree(me->d_geo);
  cudaFree(me->d_geo32);
  cudaFree(me->d_unique_map);
  cudaFree(me->d_owner);
  cudaFree(me->d_owner_mp);
  cudaFree(me->d_chunks);
  cudaFree(me->d_ghosts);
  me->d_ghosts = nullptr;
  cudaFree(me->d_u4[0]);
  cudaFree(me->d_u4[1]);
  cudaFree(me->d_status);
  cudaFree(me->d_acc_T);
  cudaFree(me->d_acc_U);
  cudaFree(me->d_adj_stat);
  cudaFree(me->d_adj_kexp);
  me->d_acc_T = me->d_acc_U = me->d_adj_stat = nullptr;
  me->d_adj_kexp = nullptr;
  cudaFree(const_cast<double*>(me->blend.sec));
  me->blend.sec = nullptr;
  cudaFree(me->d_dtab);
  cudaFree(me->d_dtab_el);
  cudaFree(me->d_dtab32);
  cudaFree(me->d_dwtab);
  cudaFree(me->d_dwtab32);
  cudaFree(me->d_dvec32);
  me->d_dtab_el = me->d_dtab32 = me->d_dwtab = me->d_dwtab32 = me->d_dvec32 = nullptr;
  cudaFree(me->d_dbnd_s);
  cudaFree(me->d_dact);
  cudaFree(me->d_dslot_owner);
  me->d_dbnd_s = me->d_dact = nullptr;
  me->d_dslot_owner = nullptr;
  cudaFree(me->d_dnodes);
  cudaFree(me->d_ditems);
  me->d_dnodes = nullptr;
  me->d_ditems = nullptr;
  cudaFree(me->d_drow_off);
  cudaFree(me->d_drow_col);
  cudaFree(me->d_drow_w);
  cudaFree(me->d_drow_w32);
  cudaFree(me->d_drow_copy_off);
  cudaFree(me->d_drow_copies);
  me->d_drow_off = me->d_drow_col = me->d_drow_copy_off = me->d_drow_copies = nullptr;
  me->d_drow_w = me->d_drow_w32 = nullptr;
  cudaFree(me->d_dcells);
  cudaFree(me->d_dcellv);
  cudaFree(me->d_dfold_off);
  cudaFree(me->d_dfold_slots);
  cudaFree(me->d_dfbnd);
  me->d_dfbnd = nullptr;
  me->d_dcellv = nullptr;
  me->d_dfold_off = me->d_dfold_slots = nullptr;
  cudaFree(me->d_dys);
  me->d_dys = nullptr;
  cudaFree(me->d_dvec);
  cudaFree(me->d_dpart);
  cudaFree(me->d_dscal);
  me->d_dtab = me->d_dvec = nullptr;
  me->d_dcells = nullptr;
  me->d_dpart = me->d_dscal = nullptr;
  me->d_geo = nullptr;
  me->d_geo32 = nullptr;
  me->d_unique_map = me->d_owner = me->d_owner_mp = nullptr;
  me->d_chunks = nullptr;
  me->d_u4[0] = me->d_u4[1] = nullptr;
  me->d_status = nullptr;
}

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

}  // namespace

namespace elm {
// Launch arguments shared by every per-node kernel of a mesh: tables, sizes,
// the current velocity and the step constants for (dt, n_sub).
AdvectArgs make_args(const elm_mesh_s* me, double dt, int n_sub) {
  elm::AdvectArgs a{};
  a.geo = me->d_geo;
  a.geo32 = me->d_geo32;
  a.n_macros = int32_t(me->n_macros);
  a.N = me->N;
  a.npm = me->npm;
  a.n_storage = me->n_storage;
  for (int r = 0; r < 3; ++r) {
    a.lo[r] = me->lo[r];
    a.hi[r] = me->hi[r];
  }
  a.u_old = me->steady ? me->d_u4[1] : me->d_u4[0];
  a.u_new = me->d_u4[1];
  a.steady = me->steady;
  a.dt = dt;
  a.n_sub = n_sub;
  a.status = me->d_status;
  a.unique_map = me->d_unique_map;
  a.owner_mp = me->d_owner_mp;
  a.chunks = me->d_chunks;
  a.n_chunks = int(me->n_chunks);
  a.ghosts = me->d_ghosts;
  a.n_ghosts = int(me->ghosts.size());
  a.skip_ghosts = 1;
  a.order = me->order;
  a.blend = me->blend;
  const double h = dt / n_sub;
  a.k64 = {h, 0.5 * h, h / 6.0, dt, 1.0 / me->M, double(me->N), {0, 0, 0}, {0, 0, 0}};
  a.k32 = {float(h), float(0.5 * h), float(h / 6.0), float(dt), float(1.0 / me->M), float(me->N),
           {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < 3; ++r) {
    a.k64.lo[r] = me->lo[r];
    a.k64.hi[r] = me->hi[r];
    a.k32.lo[r] = float(me->lo[r]);
    a.k32.hi[r] = float(me->hi[r]);
  }
  return a;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace elm

using elm::make_args;

extern "C" {

elm_status elm_mesh_create(int dim, int64_t n_vertices, const double* vertex_xyz, int64_t n_macros,
                           const int64_t* macro_vertices, int level, int precision, elm_mesh* out) {
  if (!out) return fail(ELM_ERR_ARG, "elm_mesh_create: out is null");
  if (dim != 2 && dim != 3) return fail(ELM_ERR_ARG, "elm_mesh_create: dim must be 2 or 3");
  if (n_vertices <= 0 || !vertex_xyz) return fail(ELM_ERR_ARG, "elm_mesh_create: no vertices");
  if (n_macros <= 0 || !macro_vertices) return fail(ELM_ERR_ARG, "elm_mesh_create: no macros");
  if (n_macros > (int64_t(1) << 30)) return fail(ELM_ERR_ARG, "elm_mesh_create: too many macros");
  const bool host_only = (precision & ELM_HOST_ONLY) != 0;
  const bool with_adjoint = (precision & ELM_ADJOINT) != 0;
  const int order = (precision & ELM_P1) != 0 ? 1 : 2;
  const bool with_diffusion = (precision & ELM_DIFFUSION) != 0;
  const bool with_staging = (precision & ELM_HOST_STAGING) != 0;
  precision &= ~(ELM_HOST_ONLY | ELM_ADJOINT | ELM_P1 | ELM_DIFFUSION | ELM_HOST_STAGING);
  if (precision != ELM_FP64 && precision != ELM_FP32)
    return fail(ELM_ERR_ARG, "elm_mesh_create: precision must be ELM_FP64 or ELM_FP32");
  // P1 puts one node lattice point per micro vertex, so it can go one level
  // finer than P2 for the same lattice (at most 2^10 points per edge in 2D,
  // 2^8 in 3D).
  const int max_level = (dim == 2 ? 9 : 7) + (order == 1 ? 1 : 0);
  if (level < 0 || level > max_level)
    return fail(ELM_ERR_ARG, "elm_mesh_create: level out of range (0.." + std::to_string(max_level) + ")");
  {
    // the kernels index storage slots with 32-bit integers (int32 storage)
    const int64_t M = int64_t(order) << level;
    const int64_t npm = dim == 3 ? (M + 1) * (M + 2) * (M + 3) / 6 : (M + 1) * (M + 2) / 2;
    if (n_macros * npm >= (int64_t(1) << 31))
      return fail(ELM_ERR_ARG, "elm_mesh_create: more than 2^31 - 1 storage nodes");
  }
  elm_mesh_s* me = new (std::nothrow) elm_mesh_s();
  if (!me) return fail(ELM_ERR_ARG, "elm_mesh_create: out of host memory");
  me->host_only = host_only;
  me->with_adjoint = with_adjoint;
  me->order = order;
  me->with_diffusion = with_diffusion;
  if (!host_only) {
    cudaError_t e = cudaGetDevice(&me->device);
    if (e != cudaSuccess) {
      delete me;
      return cuda_fail(e, "elm_mesh_create");
    }
  }
  std::string err;
  elm_status s;
  try {
    s = elm::build_mesh(dim, n_vertices, vertex_xyz, n_macros, macro_vertices, level, precision, me, &err);
    if (s == ELM_OK && with_staging && !host_only) s = elm::setup_host_staging(me, &err);
  } catch (const std::bad_alloc&) {
    s = ELM_ERR_ARG;
    err = "out of host memory";
  }
  if (s != ELM_OK) {
    if (!host_only) free_tables(me);
    delete me;
    return fail(s, "elm_mesh_create: " + err);
  }
  *out = me;
  return ELM_OK;
}

elm_status elm_mesh_destroy(elm_mesh me) {
  if (!me) return ELM_OK;
  if (!me->host_only) {
    DeviceGuard g(me->device);
    free_tables(me);
  }
  delete me;
  return ELM_OK;
}

int64_t elm_mesh_num_nodes(elm_mesh me) { return me ? me->n_storage : 0; }

int64_t elm_mesh_num_unique(elm_mesh me) { return me ? me->n_unique : 0; }

namespace {
// Phi of the annulus blending on the host (the kernels' formula: the sector of
// x's polar angle, lam from x parallel to (1 - lam) e_k + lam e_{k+1}, then
// rho e(theta_k + lam delta)).
void blend_point(const elm::BlendArgs& b, const std::vector<double>& sec, double* x) {
  const double t = (std::atan2(x[1], x[0]) - b.theta0) / b.delta;
  int k = int(std::floor(t)) % b.nsec;
  if (k < 0) k += b.nsec;
  const double e0 = sec[2 * k], e1 = sec[2 * k + 1], f0 = sec[2 * k + 2], f1 = sec[2 * k + 3];
  const double ck = e0 * x[1] - e1 * x[0], ck1 = f0 * x[1] - f1 * x[0];
  const double lam = ck / (ck - ck1);
  const double p0 = (1.0 - lam) * e0 + lam * f0, p1 = (1.0 - lam) * e1 + lam * f1;
  const double rho = std::sqrt(x[0] * x[0] + x[1] * x[1]) / std::sqrt(p0 * p0 + p1 * p1);
  const double th = b.theta0 + (double(k) + lam) * b.delta;
  x[0] = rho * std::cos(th);
  x[1] = rho * std::sin(th);
}

std::vector<double> sector_table(int n, double theta0) {
  std::vector<double> sec(2 * (n + 1));
  const double delta = 2.0 * 3.14159265358979323846 / n;
  for (int k = 0; k <= n; ++k) {
    sec[2 * k] = std::cos(theta0 + (k % n) * delta);
    sec[2 * k + 1] = std::sin(theta0 + (k % n) * delta);
  }
  return sec;
}
}  // namespace

elm_status elm_mesh_node_coords(elm_mesh me, double* host_out) {
  if (!me || !host_out) return fail(ELM_ERR_ARG, "elm_mesh_node_coords: null argument");
  const int d = me->dim;
  const double invM = 1.0 / me->M;
  const bool blended = me->blend.nsec > 0;
  const std::vector<double> sec = blended ? sector_table(me->blend.nsec, me->blend.theta0) : std::vector<double>();
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const elm::MacroGeo& g = me->geo[m];
    int64_t slot = m * me->npm;
    int p[3] = {0, 0, 0};
    auto emit = [&]() {
      for (int r = 0; r < d; ++r) {
        double x = g.v0[r];
        for (int c = 0; c < d; ++c) x += g.J[r * 3 + c] * (p[c] * invM);
        host_out[slot * d + r] = x;
      }
      if (blended) blend_point(me->blend, sec, host_out + slot * d);
      ++slot;
    };
    if (d == 2) {
      for (p[0] = 0; p[0] <= me->M; ++p[0])
        for (p[1] = 0; p[1] <= p[0]; ++p[1]) emit();
    } else {
      for (p[0] = 0; p[0] <= me->M; ++p[0])
        for (p[1] = 0; p[1] <= p[0]; ++p[1])
          for (p[2] = 0; p[2] <= p[1]; ++p[2]) emit();
    }
  }
  return ELM_OK;
}

elm_status elm_mesh_unique_map(elm_mesh me, int64_t* host_out) {
  if (!me || !host_out) return fail(ELM_ERR_ARG, "elm_mesh_unique_map: null argument");
  std::memcpy(host_out, me->unique_map.data(), sizeof(int64_t) * me->n_storage);
  return ELM_OK;
}

elm_status elm_to_storage(elm_mesh me, const void* unique_dev, void* storage_dev, int ncomp, void* stream) {
  if (!me || !unique_dev || !storage_dev || ncomp < 1 || ncomp > 16)
    return fail(ELM_ERR_ARG, "elm_to_storage: invalid argument");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_to_storage: host-only mesh");
  DeviceGuard g(me->device);
  cudaError_t e = elm::launch_gather(me->precision, unique_dev, storage_dev, me->d_unique_map, me->n_storage,
                                     ncomp, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ELM_OK : cuda_fail(e, "elm_to_storage");
}

elm_status elm_to_unique(elm_mesh me, const void* storage_dev, void* unique_dev, int ncomp, void* stream) {
  if (!me || !unique_dev || !storage_dev || ncomp < 1 || ncomp > 16)
    return fail(ELM_ERR_ARG, "elm_to_unique: invalid argument");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_to_unique: host-only mesh");
  DeviceGuard g(me->device);
  cudaError_t e = elm::launch_gather(me->precision, storage_dev, unique_dev, me->d_owner, me->n_unique, ncomp,
                                     static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ELM_OK : cuda_fail(e, "elm_to_unique");
}

elm_status elm_set_velocity(elm_mesh me, const void* u_old_dev, const void* u_new_dev, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_set_velocity: null mesh");
  if (!u_old_dev || !u_new_dev) return fail(ELM_ERR_ARG, "elm_set_velocity: null velocity");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_set_velocity: host-only mesh");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool steady = u_old_dev == u_new_dev;
  cudaError_t e = elm::launch_pack_velocity(me->precision, me->dim, u_new_dev, me->d_u4[1], me->n_storage, s);
  if (e == cudaSuccess && !steady)
    e = elm::launch_pack_velocity(me->precision, me->dim, u_old_dev, me->d_u4[0], me->n_storage, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_set_velocity");
  me->steady = steady;
  me->have_velocity = true;
  return ELM_OK;
}

elm_status elm_shift_velocity(elm_mesh me, const void* u_old_dev, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_shift_velocity: null mesh");
  if (!u_old_dev) return fail(ELM_ERR_ARG, "elm_shift_velocity: null velocity");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_shift_velocity: host-only mesh");
  if (!me->have_velocity) return fail(ELM_ERR_STATE, "elm_shift_velocity: elm_set_velocity has not been called");
  DeviceGuard g(me->device);
  // the current u_old's records (d_u4[0], or d_u4[1] when steady) become
  // u_new's; the other buffer receives the new u_old
  if (!me->steady) std::swap(me->d_u4[0], me->d_u4[1]);
  cudaError_t e = elm::launch_pack_velocity(me->precision, me->dim, u_old_dev, me->d_u4[0], me->n_storage,
                                            static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "elm_shift_velocity");
  me->steady = false;
  return ELM_OK;
}

elm_status elm_advect(elm_mesh me, const void* T_old_dev, void* T_new_dev, double dt, int n_sub, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_advect: null mesh");
  if (!T_old_dev || !T_new_dev) return fail(ELM_ERR_ARG, "elm_advect: null temperature buffer");
  if (!std::isfinite(dt) || dt < 0.0) return fail(ELM_ERR_ARG, "elm_advect: dt must be finite and >= 0");
  if (n_sub < 1 || n_sub > elm::kMaxSub)
    return fail(ELM_ERR_ARG, "elm_advect: n_sub must be in 1.." + std::to_string(elm::kMaxSub));
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_advect: host-only mesh");
  if (!me->have_velocity) return fail(ELM_ERR_STATE, "elm_advect: elm_set_velocity has not been called");
  if (ranges_overlap(T_old_dev, T_new_dev, elem_size(me) * size_t(me->n_storage)))
    return fail(ELM_ERR_ARG, "elm_advect: T_old and T_new overlap");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  elm::AdvectArgs a = make_args(me, dt, n_sub);
  a.T_old = T_old_dev;
  a.T_new = T_new_dev;
  cudaError_t e = elm::launch_advect(me->dim, me->precision, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_advect");
  return ELM_OK;
}

elm_status elm_advect_adjoint(elm_mesh me, const void* T_old_dev, const void* gT_new_dev, void* gT_old_dev,
                              void* gU_old_dev, void* gU_new_dev, double dt, int n_sub, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_advect_adjoint: null mesh");
  if (!T_old_dev || !gT_new_dev || !gT_old_dev || !gU_old_dev)
    return fail(ELM_ERR_ARG, "elm_advect_adjoint: null buffer");
  if (!std::isfinite(dt) || dt < 0.0) return fail(ELM_ERR_ARG, "elm_advect_adjoint: dt must be finite and >= 0");
  if (n_sub < 1 || n_sub > elm::kMaxAdjointSub)
    return fail(ELM_ERR_ARG, "elm_advect_adjoint: n_sub must be in 1.." + std::to_string(elm::kMaxAdjointSub));
  if (me->host_only || !me->with_adjoint)
    return fail(ELM_ERR_STATE, "elm_advect_adjoint: mesh was created without ELM_ADJOINT");
  if (!me->have_velocity) return fail(ELM_ERR_STATE, "elm_advect_adjoint: elm_set_velocity has not been called");
  if (me->steady && gU_new_dev)
    return fail(ELM_ERR_ARG, "elm_advect_adjoint: steady velocity: pass gU_new = NULL (gU_old gets the gradient)");
  const size_t bytes = elem_size(me) * size_t(me->n_storage);
  if (ranges_overlap(gT_new_dev, gT_old_dev, bytes)) return fail(ELM_ERR_ARG, "elm_advect_adjoint: gT_new and gT_old overlap");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  elm::AdvectArgs a = make_args(me, dt, n_sub);
  a.T_old = T_old_dev;
  a.T_new = nullptr;
  const elm::AdjointBuffers b{me->d_acc_T,  me->d_acc_U, me->d_adj_stat, me->d_adj_stat + 3 * me->n_storage,
                              me->d_adj_kexp, me->d_owner, me->d_ghosts, int(me->ghosts.size())};
  cudaError_t e = elm::launch_adjoint(me->dim, me->precision, a, b, gT_new_dev, gT_old_dev, gU_old_dev,
                                      me->steady ? nullptr : gU_new_dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_advect_adjoint");
  return ELM_OK;
}

elm_status elm_trace(elm_mesh me, const void* D_in_dev, void* D_out_dev, double dt, int n_sub, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_trace: null mesh");
  if (!D_out_dev) return fail(ELM_ERR_ARG, "elm_trace: null output buffer");
  if (!std::isfinite(dt) || dt < 0.0) return fail(ELM_ERR_ARG, "elm_trace: dt must be finite and >= 0");
  if (n_sub < 1 || n_sub > elm::kMaxSub)
    return fail(ELM_ERR_ARG, "elm_trace: n_sub must be in 1.." + std::to_string(elm::kMaxSub));
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_trace: host-only mesh");
  if (!me->have_velocity) return fail(ELM_ERR_STATE, "elm_trace: elm_set_velocity has not been called");
  if (D_in_dev && ranges_overlap(D_in_dev, D_out_dev, elem_size(me) * size_t(me->n_storage) * me->dim))
    return fail(ELM_ERR_ARG, "elm_trace: D_in and D_out overlap");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  elm::AdvectArgs a = make_args(me, dt, n_sub);
  a.mode = 1;
  a.D_in = D_in_dev;
  a.D_out = D_out_dev;
  cudaError_t e = elm::launch_advect(me->dim, me->precision, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_trace");
  return ELM_OK;
}

elm_status elm_trace_eval(elm_mesh me, const void* D_dev, const void* T_src_dev, void* T_dst_dev, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_trace_eval: null mesh");
  if (!D_dev || !T_src_dev || !T_dst_dev) return fail(ELM_ERR_ARG, "elm_trace_eval: null buffer");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_trace_eval: host-only mesh");
  if (ranges_overlap(T_src_dev, T_dst_dev, elem_size(me) * size_t(me->n_storage)))
    return fail(ELM_ERR_ARG, "elm_trace_eval: T_src and T_dst overlap");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  elm::AdvectArgs a = make_args(me, 0.0, 1);
  a.mode = 2;
  a.D_in = D_dev;
  a.T_old = T_src_dev;
  a.T_new = T_dst_dev;
  cudaError_t e = elm::launch_advect(me->dim, me->precision, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_trace_eval");
  return ELM_OK;
}

elm_status elm_mesh_set_annulus(elm_mesh me, double r_min, double r_max, int n_sectors, double theta0) {
  if (!me) return fail(ELM_ERR_ARG, "elm_mesh_set_annulus: null mesh");
  if (me->dim != 2 || me->precision != ELM_FP64)
    return fail(ELM_ERR_ARG, "elm_mesh_set_annulus: blending is built for 2D FP64 meshes");
  if (me->with_adjoint) return fail(ELM_ERR_ARG, "elm_mesh_set_annulus: not combinable with ELM_ADJOINT");
  if (me->blend.nsec > 0) return fail(ELM_ERR_STATE, "elm_mesh_set_annulus: the mesh is blended already");
  if (n_sectors < 3 || n_sectors > 4096 || !std::isfinite(theta0) || !(r_min > 0.0) || !(r_max > r_min) ||
      !std::isfinite(r_max))
    return fail(ELM_ERR_ARG, "elm_mesh_set_annulus: need 3 <= n_sectors <= 4096 and 0 < r_min < r_max");
  // every macro: vertices on circles within [r_min, r_max] at sector angles,
  // spanning exactly one sector
  const double delta = 2.0 * 3.14159265358979323846 / n_sectors;
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const elm::MacroGeo& g = me->geo[m];
    int ks[3];
    for (int v = 0; v <= 2; ++v) {
      double x[2] = {g.v0[0], g.v0[1]};
      for (int c = 0; c < v; ++c) {
        x[0] += g.J[0 * 3 + c];
        x[1] += g.J[1 * 3 + c];
      }
      const double r = std::sqrt(x[0] * x[0] + x[1] * x[1]);
      const double t = (std::atan2(x[1], x[0]) - theta0) / delta;
      const double kr = std::nearbyint(t);
      if (r < r_min * (1 - 1e-12) || r > r_max * (1 + 1e-12) || std::fabs(t - kr) > 1e-9)
        return fail(ELM_ERR_TOPOLOGY, "elm_mesh_set_annulus: macro " + std::to_string(m) +
                                          " has a vertex off the ring's sector rays or radii");
      ks[v] = ((int(kr) % n_sectors) + n_sectors) % n_sectors;
    }
    int lo = ks[0];
    bool one_sector = false;
    for (int v = 0; v <= 2 && !one_sector; ++v) {
      lo = ks[v];
      bool ok = true;
      for (int w = 0; w <= 2; ++w) ok = ok && (ks[w] == lo || ks[w] == (lo + 1) % n_sectors);
      bool has_lo = false, has_hi = false;
      for (int w = 0; w <= 2; ++w) {
        has_lo = has_lo || ks[w] == lo;
        has_hi = has_hi || ks[w] == (lo + 1) % n_sectors;
      }
      one_sector = ok && has_lo && has_hi;
    }
    if (!one_sector)
      return fail(ELM_ERR_TOPOLOGY, "elm_mesh_set_annulus: macro " + std::to_string(m) + " does not span one sector");
  }
  const std::vector<double> sec = sector_table(n_sectors, theta0);
  double* d_sec = nullptr;
  if (!me->host_only) {
    DeviceGuard g(me->device);
    cudaError_t e = cudaMalloc((void**)&d_sec, sizeof(double) * sec.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_sec, sec.data(), sizeof(double) * sec.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d_sec);
      return cuda_fail(e, "elm_mesh_set_annulus");
    }
  }
  me->blend.sec = d_sec;
  me->blend.nsec = n_sectors;
  me->blend.theta0 = theta0;
  me->blend.delta = delta;
  me->blend.rmin = r_min;
  me->blend.rmax = r_max;
  if (me->with_diffusion && !me->host_only) {
    DeviceGuard g(me->device);
    std::string err;
    const elm_status st = elm::build_diffusion_blended(me, &err);
    if (st != ELM_OK) return fail(st, "elm_mesh_set_annulus: " + err);
  }
  return ELM_OK;
}

elm_status elm_get_status(elm_mesh me, void* stream) {
  if (!me) return fail(ELM_ERR_ARG, "elm_get_status: null mesh");
  if (me->host_only) return fail(ELM_ERR_STATE, "elm_get_status: host-only mesh");
  DeviceGuard g(me->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned flags = 0;
  cudaError_t e = cudaMemcpyAsync(&flags, me->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(me->d_status, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(e, "elm_get_status");
  if (flags & elm::kFlagWalkLimit)
    return fail(ELM_ERR_WALK_LIMIT, "a point needed more than the macro-walk limit of hops");
  if (flags & elm::kFlagNonFinite) return fail(ELM_ERR_NONFINITE, "a velocity or result value was not finite");
  return ELM_OK;
}

const char* elm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
