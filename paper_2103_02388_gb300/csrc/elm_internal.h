// elm_internal.h -- internal types shared by the host mesh builder, the C ABI
// and the CUDA kernels of libelm.so.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "elm.h"

namespace elm {

constexpr int kMaxHops = 32;           // macro walk limit per location
constexpr unsigned kFlagWalkLimit = 1u;
constexpr unsigned kFlagNonFinite = 2u;

// Affine data of one macro simplex (Sec. 2.1).  The vertices P_0..P_d are
// taken in ascending global id; the reference Kuhn simplex
// {1 >= s_1 >= .. >= s_d >= 0} is mapped by x = P_0 + J s with
// J = [P_1 - P_0 | P_2 - P_1 | P_3 - P_2], and the level-L lattice coordinate
// is q = N s = NJinv (x - P_0), N = 2^L.
// Lattice frame change across face k of a macro m to its neighbour mm:
// q_mm = A q_m + b with A = J_mm^{-1} J_m and b = N J_mm^{-1} (v0_m - v0_mm).
// Stored when A and b are exactly integers (bit k of `exact`), as for macros
// that are lattice-congruent images of one another (the Kuhn tetrahedra of a
// cube, the two triangles of a square); a point on the lattice of m with
// half-integer coordinates then changes frame in exact integer-valued
// arithmetic instead of recomputing its position.
struct FaceXform {
  int8_t A[4][9];    // row-major d x d per face
  int32_t b[4][3];
  int32_t exact;     // bit k: face k's transform is stored
};

struct MacroGeo {
  double v0[3];
  double J[9];       // row-major d x d (leading d x d block used in 2D)
  double NJinv[9];   // row-major, N * J^{-1}
  int32_t nb[4];     // macro across the face opposite local vertex k; -1 = boundary
  FaceXform x;
};

// FP32 copy of the macro data, used by the FP32 kernel.  Each FP64 value x is
// also kept as a pair (hi, lo) with hi = float(x), lo = float(x - hi), so that
// the rare start-node frame changes can be computed in double-float
// arithmetic on the FP32 pipe.
struct MacroGeo32 {
  float NJinv[9];
  float J[9];
  float v0[3];
  int32_t nb[4];
  float NJinv_lo[9];
  float J_lo[9];
  float v0_lo[3];
  FaceXform x;
};

// Launch constants in the kernel's working precision, computed once on the
// host (a per-thread FP64 division or conversion costs dozens of cycles on
// this GPU's narrow FP64 pipe).
template <class R>
struct StepConsts {
  R h, h2, h6;     // substep, half substep, substep / 6
  R dt;
  R invM;          // 1 / M, M = order * 2^L (the node lattice)
  R Nf;            // 2^L
  R lo[3], hi[3];  // bounding box
};

// Blending onto an annulus (Sec. 2.1, blending map Phi; elm_mesh_set_annulus):
// a 2D ring mesh of nsec sectors with vertices at the angles theta0 + k delta
// on circles, mapped sector by sector in polar form (see tracer.cuh).
// nsec = 0: no blending (Phi = Id).
struct BlendArgs {
  const double* sec = nullptr;  // unit vectors e_k at theta0 + k delta, k = 0..nsec ([nsec + 1][2])
  int nsec = 0;
  double theta0 = 0.0, delta = 0.0, rmin = 0.0, rmax = 0.0;
};

// Everything a kernel launch needs, passed by value.
struct AdvectArgs {
  const MacroGeo* geo;     // [n_macros]
  const MacroGeo32* geo32; // [n_macros]
  int32_t n_macros;
  int32_t N;               // 2^L
  int64_t npm;             // storage nodes per macro
  int64_t n_storage;
  double lo[3], hi[3];     // bounding box (domain clamp)
  const void* u_old;      // packed velocity records [n, 4] (x, y[, z], 0)
  const void* u_new;
  int steady;              // u_old == u_new
  const void* T_old;
  void* T_new;
  double dt;
  int n_sub;
  unsigned* status;
  const int64_t* unique_map;  // storage slot -> unique id
  const int64_t* owner_mp;    // unique id -> owner record (pack_owner)
  const int4* chunks;         // (macro, p1, first index in slab, count) per thread block
  int n_chunks;
  // Interface copies (a5, ghost copy): with skip_ghosts the per-node kernel
  // computes each node once, in its owner's slot, and a copy pass then fills
  // the other storage copies from the (ghost slot, owner slot) pairs.
  const int2* ghosts = nullptr;
  int n_ghosts = 0;
  int skip_ghosts = 0;
  int order = 2;              // element order: 1 (P1) or 2 (P2)
  int mode = 0;               // per-node work (NodeMode in tracer.cuh): step, trace, evaluation
  const void* D_in = nullptr; // departure offsets [n, dim] (trace / evaluation)
  void* D_out = nullptr;
  BlendArgs blend;
  StepConsts<float> k32;
  StepConsts<double> k64;
};

// Host-buffer step (elm_advect_host, ELM_HOST_STAGING): two sets of device
// staging buffers used by alternate calls, so that the host-to-device copy of
// one call runs while the previous call computes and copies its result back.
// The step of a call is launched in kHostParts pieces (contiguous runs of the
// work list, which cover contiguous storage ranges), and each piece's result
// goes back to the host as soon as that piece is done.
constexpr int kHostParts = 4;
struct HostStaging {
  void* u[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [set][old, new]: velocity [n, dim]
  void* T_old[2] = {nullptr, nullptr};
  void* T_new[2] = {nullptr, nullptr};
  cudaStream_t h2d = nullptr, d2h = nullptr;   // non-blocking copy streams
  cudaEvent_t ev_h2d[2] = {nullptr, nullptr};  // inputs of the set are on the device
  cudaEvent_t ev_part[2][kHostParts] = {};     // piece p of the set's step is done
  cudaEvent_t ev_d2h[2] = {nullptr, nullptr};  // the set's result is on the host
  cudaEvent_t ev_free[2] = {nullptr, nullptr}; // the set may be overwritten
  int next = 0;                                // set of the next call
  const char* out_ptr[2] = {nullptr, nullptr}; // host result range of each set's last call
  size_t out_bytes[2] = {0, 0};
  int64_t part_chunk[kHostParts + 1] = {};     // piece p: chunks [part_chunk[p], part_chunk[p+1])
  int64_t part_slot[kHostParts + 1] = {};      // and storage slots [part_slot[p], part_slot[p+1])
  int64_t part_ghost[kHostParts + 1] = {};     // and ghost pairs [part_ghost[p], part_ghost[p+1])
};

}  // namespace elm

struct elm_mesh_s {
  int dim = 0, level = 0, N = 0, M = 0, precision = ELM_FP64;
  int order = 2;                     // element order (P1 / P2); M = order * N
  elm::BlendArgs blend;              // annulus blending (nsec > 0), device sector table in blend.sec
  bool host_only = false;
  int64_t n_macros = 0, npm = 0, n_storage = 0, n_unique = 0, n_ghost = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  std::vector<elm::MacroGeo> geo;
  std::vector<int64_t> unique_map;   // storage slot -> unique id
  std::vector<int64_t> owner;        // unique id -> owner storage slot
  int device = 0;
  // device tables
  elm::MacroGeo* d_geo = nullptr;
  elm::MacroGeo32* d_geo32 = nullptr;
  int64_t* d_unique_map = nullptr;
  int64_t* d_owner = nullptr;
  int64_t* d_owner_mp = nullptr;     // unique id -> owner record (pack_owner)
  int4* d_chunks = nullptr;          // work list: one block-sized run of a slab each
  int64_t n_chunks = 0;
  std::vector<int4> chunks;          // host copy of the work list
  std::vector<int2> ghosts;          // (ghost slot, owner slot), ascending ghost slot
  int2* d_ghosts = nullptr;
  elm::HostStaging* staging = nullptr;  // ELM_HOST_STAGING
  void* d_u4[2] = {nullptr, nullptr};  // packed velocity records u_old, u_new
  bool have_velocity = false;
  bool steady = true;
  // adjoint scratch (ELM_ADJOINT)
  bool with_adjoint = false;
  unsigned long long* d_acc_T = nullptr;
  unsigned long long* d_acc_U = nullptr;
  unsigned long long* d_adj_stat = nullptr;  // [2][3 n]: largest |contribution| bits, count
  int* d_adj_kexp = nullptr;                 // [3 n]
  unsigned* d_status = nullptr;
  // diffusion solver (ELM_DIFFUSION): element tables and stencil weights per
  // macro, the interior node lists of the stencil pass, the assembled rows of
  // the face nodes, masks and CG vectors in the storage layout, reduction
  // space
  bool with_diffusion = false;
  void* d_dtab = nullptr;
  void* d_dtab_el = nullptr;         // blended meshes: per-simplex mass and stiffness
  void* d_dtab32 = nullptr;          // FP64 meshes: FP32 copy of the tables (inner solves)
  void* d_dwtab = nullptr;           // node-centred stencil weights per macro: [mass | stiffness][entries]
  void* d_dwtab32 = nullptr;         // FP64 meshes: FP32 copy of the stencil weights
  void* d_dvec32 = nullptr;          // FP64 meshes: FP32 vectors of the inner solves
  std::vector<uint8_t> dbnd;         // per unique node: Dirichlet boundary
  uint8_t* d_dbnd_s = nullptr;       // per storage slot: Dirichlet boundary
  uint8_t* d_dact = nullptr;         // per storage slot: owner copy of an interior unknown (dot products)
  int64_t* d_dslot_owner = nullptr;  // per storage slot: the owner slot of its node
  // interior nodes (node-centred stencil): packed lattice points by macro and
  // class, warp items (macro, class, first node, count), 4 per block (one macro)
  uint32_t* d_dnodes = nullptr;
  int4* d_ditems = nullptr;
  int64_t n_ditems = 0;
  int n_dsm = 0;                     // SMs of the device (grids of the operator passes)
  // face nodes off the Dirichlet boundary (assembled rows): row r has entries
  // [row_off[r], row_off[r + 1]) of (column slot, mass weight, stiffness
  // weight) and writes its value to the copies [copy_off[r], copy_off[r + 1])
  int64_t n_drows = 0;
  int64_t n_dnnz = 0;
  int* d_drow_off = nullptr;
  int* d_drow_col = nullptr;
  void* d_drow_w = nullptr;          // [2][nnz]: mass, then stiffness weights (mesh precision)
  void* d_drow_w32 = nullptr;        // FP64 meshes: FP32 copy
  int* d_drow_copy_off = nullptr;
  int* d_drow_copies = nullptr;
  // blended meshes (per-simplex tables): the cell pass over every cell and
  // its fold into every node
  int4* d_dcells = nullptr;          // (macro, first cell, count, colour) chunks of the cell pass
  int4* d_dcellv = nullptr;          // cells (c0, c1, c2) in colour, then macro order
  int64_t n_cell_chunks = 0;
  int64_t n_dface = 0;               // fold nodes (every unique node)
  int* d_dfold_off = nullptr;        // fold node f -> its storage copies, ascending slot: [off[f], off[f + 1])
  int* d_dfold_slots = nullptr;
  uint8_t* d_dfbnd = nullptr;        // per fold node: Dirichlet boundary
  void* d_dys = nullptr;             // blended meshes: colour accumulators per storage slot
  int64_t n_boundary = 0;
  void* d_dvec = nullptr;
  double* d_dpart = nullptr;
  double* d_dscal = nullptr;
};

namespace elm {

// Sets the thread-local message returned by elm_last_error (api.cpp).
void set_last_error(const std::string& msg);

// Vectors of the diffusion solver (x, r, z, p, q, b, inverse diagonal), and
// the FP32 vectors of the inner solves on FP64 meshes (r, z, p, q, d, inverse
// diagonal).
constexpr int kDiffVectors = 7;
constexpr int kDiffVectors32 = 6;

// Diffusion solver set-up at mesh creation (diffusion.cu), and the per-simplex
// tables of a blended mesh (at elm_mesh_set_annulus).
elm_status build_diffusion(elm_mesh_s* me, std::string* err);
elm_status build_diffusion_blended(elm_mesh_s* me, std::string* err);

// Host-buffer step set-up and tear-down (host_path.cpp).
elm_status setup_host_staging(elm_mesh_s* me, std::string* err);
void free_host_staging(elm_mesh_s* me);

// Launch arguments of a per-node kernel of the mesh for a step (dt, n_sub):
// tables, sizes, the current velocity and the step constants (api.cpp).
AdvectArgs make_args(const elm_mesh_s* me, double dt, int n_sub);

// Host mesh construction (mesh.cpp).
elm_status build_mesh(int dim, int64_t nv, const double* xyz, int64_t nm, const int64_t* mv,
                      int level, int precision, elm_mesh_s* me, std::string* err);

// Packed P2 node index of lattice point p inside a macro (storage layout).
inline int64_t packed_index_host(int dim, const int* p) {
  if (dim == 3)
    return int64_t(p[0]) * (p[0] + 1) * (p[0] + 2) / 6 + int64_t(p[1]) * (p[1] + 1) / 2 + p[2];
  return int64_t(p[0]) * (p[0] + 1) / 2 + p[1];
}

inline int64_t nodes_per_macro(int dim, int M) {
  return dim == 3 ? int64_t(M + 1) * (M + 2) * (M + 3) / 6 : int64_t(M + 1) * (M + 2) / 2;
}

// Kernel launchers (advect.cu).  Return a CUDA error code.
cudaError_t launch_advect(int dim, int precision, const AdvectArgs& a, cudaStream_t s);
cudaError_t launch_gather(int precision, const void* in, void* out, const int64_t* idx, int64_t n,
                          int ncomp, cudaStream_t s);
cudaError_t launch_pack_velocity(int precision, int dim, const void* u, void* u4, int64_t n, cudaStream_t s);

// Nodes per work-list chunk (and threads per block of the batched and adjoint
// kernels).  k_advect runs each chunk as kAdvectSplit blocks of kStepThreads
// threads: smaller blocks retire warp pairs independently, so a warp held up
// on a slow path keeps fewer registers idle (measured at level 7 FP32:
// 0.736 ms against 0.750 ms with one 128-thread block per chunk, and 0.81 ms
// with 32-thread blocks, which spill more).
constexpr int kAdvectThreads = 128;
constexpr int kStepThreads = 64;
constexpr int kAdvectSplit = kAdvectThreads / kStepThreads;

// ---------------------------------------------------------------------------
// Batched form: many independent meshes in one persistent launch.
// ---------------------------------------------------------------------------
// Owner record of a unique node: its owner macro and the owner's lattice
// point (p1, p2[, p3]) in 11-bit fields, enough for lattice coordinates up
// to 2047 (the largest lattice is 2^10 in 2D).
constexpr int kOwnerBits = 11;
constexpr int kOwnerMask = (1 << kOwnerBits) - 1;
__host__ __device__ inline int64_t pack_owner(int64_t macro, int p1, int p2, int p3) {
  return (macro << (3 * kOwnerBits)) | (int64_t(p1) << (2 * kOwnerBits)) | (int64_t(p2) << kOwnerBits) | p3;
}
template <int D>
__host__ __device__ inline int unpack_owner(int64_t own, int* p) {
  p[0] = int(own >> (2 * kOwnerBits)) & kOwnerMask;
  p[1] = int(own >> kOwnerBits) & kOwnerMask;
  if (D == 3) p[D - 1] = int(own) & kOwnerMask;
  return int(own >> (3 * kOwnerBits));
}

constexpr int kMaxBatch = 128;
constexpr int kMaxSub = ELM_MAX_SUBSTEPS;
constexpr int kMaxAdjointSub = ELM_MAX_ADJOINT_SUBSTEPS;

// Per instance, fixed for the batch's lifetime (device table).
struct BatchStatic {
  const MacroGeo* geo;
  const MacroGeo32* geo32;
  const int64_t* unique_map;
  const int64_t* owner_mp;
  const int4* chunks;
  unsigned* status;
  int N;
  int npm;
  int dim;
  int pad;
};

// Per instance, per call (passed by value in the kernel's parameters, so a
// captured CUDA graph replays exactly the pointers and constants given).
template <class R>
struct BatchCall {
  const void* u_old;
  const void* u_new;
  const void* T_old;
  void* T_new;
  int n_sub;
  int steady;
  StepConsts<R> K;
};

template <class R>
struct BatchParams {
  const BatchStatic* inst;
  const int4* items;  // (instance, first chunk, chunks) work list: runs of consecutive chunks of one instance
  int n_items;
  int count;
  int* counter;       // next work item; zeroed before every launch
  BatchCall<R> call[kMaxBatch];
};

// Scratch of the adjoint (allocated at mesh creation with ELM_ADJOINT).
struct AdjointBuffers {
  unsigned long long* acc_T;    // [n] 64-bit fixed-point sums
  unsigned long long* acc_U;    // [2][dim][n] (component-major)
  unsigned long long* smax;     // [3 n] per slot: largest |contribution| (value bits); T, then 2 velocity sets
  unsigned long long* scnt;     // [3 n] per slot: number of contributions
  int* kexp;                    // [3 n] per slot: scale exponent
  const int64_t* owner;         // unique id -> owner slot
  const int2* ghosts;           // (copy slot, owner slot) of every interface copy
  int n_ghosts;
};
cudaError_t launch_adjoint(int dim, int precision, const AdvectArgs& a, const AdjointBuffers& b,
                           const void* gT_new, void* gT_old, void* gU_old, void* gU_new, cudaStream_t s);

// The batched kernel of element order `order` with `min_blocks` resident
// blocks per SM reserved by its register budget (6 or 8); the interface
// copies of every instance are filled afterwards by launch_batch_ghosts from
// (instance, copy slot, owner slot) triples.
cudaError_t launch_batch32(const BatchParams<float>& p, int order, int min_blocks, int grid, cudaStream_t s);
cudaError_t launch_batch64(const BatchParams<double>& p, int order, int min_blocks, int grid, cudaStream_t s);
cudaError_t launch_batch_ghosts32(const BatchParams<float>& p, const int4* g, int n, cudaStream_t s);
cudaError_t launch_batch_ghosts64(const BatchParams<double>& p, const int4* g, int n, cudaStream_t s);

}  // namespace elm
