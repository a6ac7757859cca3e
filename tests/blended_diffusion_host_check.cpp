// blended_diffusion_host_check.cpp -- the diffusion operator of a mesh blended
// onto an annulus (csrc/diffusion.cu: blended_element_tables, the cell lists
// and fold of build_cells_and_fold, the cell pass k_apply<2, double, P, DIAG,
// true> and its fold k_fold_nodes<double, 4, MODE>) compiled with g++ and run
// on the CPU, each block's threads together (CUDA_HOST_THREADS in
// tests/cuda_host_shim.h), under AddressSanitizer and
// UndefinedBehaviorSanitizer, for a CPU check against the oracle's assembled
// blended mass and stiffness matrices (tests/test_kernel_host.py).  No GPU.
//
// The set-up code places its tables with cudaMalloc / cudaMemcpy / cudaMemset
// / cudaFree; here those four are host-memory stand-ins (malloc, memcpy,
// memset, free), so the kernels read the same tables from host memory.
//
// Input file (little-endian): int64 [n_vertices, n_macros, level, order, mode
// (0: y += scale (M + alpha A) x, 1: the CG form y = that, 0 on the Dirichlet
// boundary, with p.y summed into the CG scalars, p = x; 2: y += its
// diagonal)], doubles [alpha, scale, r_min, r_max, n_sectors, theta0], vertex
// coordinates [n_vertices * 2], macro vertices (int64), x [n_storage]
// (doubles).  Output file: y [n_storage], then p.y (doubles).  Exit status 0,
// or 1 on bad input.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace host_mem {
inline cudaError_t alloc(void** p, size_t n) {
  *p = std::malloc(n);
  return *p != nullptr ? cudaSuccess : cudaErrorMemoryAllocation;
}
template <class T>
inline cudaError_t alloc(T** p, size_t n) {
  void* q = nullptr;
  const cudaError_t e = alloc(&q, n);
  *p = static_cast<T*>(q);
  return e;
}
inline cudaError_t copy(void* d, const void* s, size_t n, cudaMemcpyKind) {
  std::memcpy(d, s, n);
  return cudaSuccess;
}
inline cudaError_t set(void* d, int v, size_t n) {
  std::memset(d, v, n);
  return cudaSuccess;
}
inline cudaError_t release(void* p) {
  std::free(p);
  return cudaSuccess;
}
}  // namespace host_mem

#define cudaMalloc host_mem::alloc
#define cudaMemcpy host_mem::copy
#define cudaMemset host_mem::set
#define cudaFree host_mem::release
#include "diffusion_front.cuh"
#undef cudaMalloc
#undef cudaMemcpy
#undef cudaMemset
#undef cudaFree

using namespace elm;

namespace {

template <class T>
bool read_n(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

template <int P, int MODE>
void apply(elm_mesh_s* me, const std::vector<double>& x, double alpha, double scale, std::vector<double>& out) {
  const size_t n = size_t(me->n_storage);
  std::vector<double> y(n, 0.0);
  Scalars sc{};
  sc.rz = 1.0;
  sc.budget = 1 << 30;
  const bool cg = MODE == kOpCg;
  const int nfb = me->n_dface > 0 ? red_blocks(me->n_dface) : 0;
  std::vector<double> part(size_t(nfb) + 1, 0.0);
  OpArgs a{me->d_dtab_el, me->d_dcells, me->d_dcellv, int(me->npm), me->N, cg ? &sc : nullptr};
  double* ys = static_cast<double*>(me->d_dys);
  constexpr bool DG = MODE == kOpDiag;
  if (me->n_cell_chunks > 0)
    host_launch(unsigned(me->n_cell_chunks), kDiffThreads,
                [&] { k_apply<2, double, P, DG, true>(a, x.data(), ys, alpha, scale); });
  if (nfb > 0)
    host_launch(unsigned(nfb), kRedThreads, [&] {
      k_fold_nodes<double, 4, MODE>(ys, y.data(), me->d_dfold_off, me->d_dfold_slots, me->d_dfbnd, me->n_dface,
                                    x.data(), part.data(), cg ? &sc : nullptr);
    });
  out = y;
  out.push_back(sc.pq);
}

template <int MODE>
void dispatch(elm_mesh_s* me, const std::vector<double>& x, double alpha, double scale, std::vector<double>& out) {
  if (me->order == 2)
    apply<2, MODE>(me, x, alpha, scale, out);
  else
    apply<1, MODE>(me, x, alpha, scale, out);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 1;
  std::vector<int64_t> hd, Mc;
  std::vector<double> ab, V, x, out;
  if (!read_n(f, hd, 5) || !read_n(f, ab, 6)) return 1;
  const int order = int(hd[3]), mode = int(hd[4]);
  if (!read_n(f, V, size_t(hd[0] * 2)) || !read_n(f, Mc, size_t(hd[1] * 3))) return 1;
  elm_mesh mesh = nullptr;
  const int prec = ELM_FP64 | ELM_HOST_ONLY | (order == 1 ? ELM_P1 : 0);
  if (elm_mesh_create(2, hd[0], V.data(), hd[1], Mc.data(), int(hd[2]), prec, &mesh) != ELM_OK ||
      elm_mesh_set_annulus(mesh, ab[2], ab[3], int(ab[4]), ab[5]) != ELM_OK) {
    std::fprintf(stderr, "mesh: %s\n", elm_last_error());
    return 1;
  }
  elm_mesh_s* me = mesh;
  if (!read_n(f, x, size_t(me->n_storage))) return 1;
  std::fclose(f);
  // the Dirichlet mask comes with the affine set-up, as at mesh creation;
  // then the blended tables, cell lists and fold, as elm_mesh_set_annulus
  // builds them
  (void)diffusion_host(me);
  std::vector<double> t;
  blended_element_tables(me, t);
  const bool ok = upload_real(&me->d_dtab_el, t, true) && build_cells_and_fold(me);
  if (ok) {
    if (mode == 0)
      dispatch<kOpAccum>(me, x, ab[0], ab[1], out);
    else if (mode == 1)
      dispatch<kOpCg>(me, x, ab[0], ab[1], out);
    else
      dispatch<kOpDiag>(me, x, ab[0], ab[1], out);
  }
  // the host copies are this program's; the mesh does not free them
  void* owned[] = {me->d_dtab_el, me->d_dcells, me->d_dcellv, me->d_dfold_off, me->d_dfold_slots, me->d_dfbnd,
                   me->d_dys};
  for (void* p : owned) std::free(p);
  me->d_dtab_el = me->d_dys = nullptr;
  me->d_dcells = me->d_dcellv = nullptr;
  me->d_dfold_off = me->d_dfold_slots = nullptr;
  me->d_dfbnd = nullptr;
  elm_mesh_destroy(mesh);
  if (!ok) {
    std::fprintf(stderr, "blended set-up failed\n");
    return 1;
  }
  FILE* g = std::fopen(argv[2], "wb");
  if (!g || std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 1;
  std::fclose(g);
  return 0;
}
