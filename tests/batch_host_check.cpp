// batch_host_check.cpp -- the batched persistent kernel (k_advect_batch,
// csrc/advect.cu) compiled with g++ and run on the CPU, each block's threads
// together (CUDA_HOST_THREADS in tests/cuda_host_shim.h), under
// AddressSanitizer / UndefinedBehaviorSanitizer or ThreadSanitizer, for a CPU
// check against the single-instance host step and the oracle
// (tests/test_kernel_host.py).  No GPU.
//
// The test writes advect_front.cuh: the part of advect.cu before its launch
// functions (the kernels, no launches).  Each instance is a host-only mesh
// with the tables the library uploads (tests/host_mesh_tables.h); the batch's
// static table, per-call parameters and work list (runs of `chunks_per_item`
// chunks of one instance) are built as elm_batch_create and elm_batch_advect
// build them (the velocity records by k_pack_velocity), and every block takes
// work items from the shared counter until the list is done.  The interface
// copies of every instance are filled afterwards by k_batch_ghost_copy, and
// k_gather reads each result back in node order (the owner copies).
//
// Input file (little-endian): int64 [count, precision (0: FP64, 1: FP32),
// chunks_per_item, blocks]; per instance int64 [dim, n_vertices, n_macros,
// level, steady, n_sub], double dt, vertex coordinates, macro vertices
// (int64), u^n, u^{n+1} [n_storage * dim], T^n [n_storage] (doubles; P2
// elements).  Output file: every instance's T^{n+1} [n_storage], in order,
// then every instance's T^{n+1} [n_unique] in node order (doubles).  Exit status 0, 1 on bad input, 2 on a device-side status flag.
#include <cstdio>
#include <memory>
#include <vector>

#include "advect_front.cuh"
#include "host_mesh_tables.h"

using namespace elm;
using elm_host_check::HostTables;
using elm_host_check::host_tables;

namespace {

template <class T>
bool read_n(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

struct Instance {
  elm_mesh_s* me = nullptr;
  HostTables h;
  int steady = 1, n_sub = 1;
  double dt = 0;
  std::vector<double> uo, un, T;
};

template <class R>
int run(std::vector<Instance>& inst, int chunks_per_item, unsigned blocks, std::vector<double>& out) {
  const int count = int(inst.size());
  std::vector<BatchStatic> st(static_cast<size_t>(count));
  std::vector<unsigned> status(static_cast<size_t>(count), 0u);
  const size_t nk = static_cast<size_t>(count);
  std::vector<std::vector<R>> un(nk), uo(nk), T(nk), Tn(nk);
  auto B = std::make_unique<BatchParams<R>>();
  std::vector<int4> items;
  for (int k = 0; k < count; ++k) {
    Instance& I = inst[size_t(k)];
    elm_mesh_s* me = I.me;
    const size_t n = size_t(me->n_storage);
    const int d = me->dim;
    un[size_t(k)].assign(n * 4, R(0));
    uo[size_t(k)].assign(n * 4, R(0));
    T[size_t(k)].assign(n, R(0));
    Tn[size_t(k)].assign(n, R(0));
    // the instance's velocity records, as elm_set_velocity packs them
    std::vector<R> vn(I.un.begin(), I.un.end()), vo(I.uo.begin(), I.uo.end());
    const unsigned pb = unsigned((n + 255) / 256);
    host_launch(pb, 256, [&] { k_pack_velocity<R>(vn.data(), un[size_t(k)].data(), int64_t(n), d); });
    host_launch(pb, 256, [&] { k_pack_velocity<R>(vo.data(), uo[size_t(k)].data(), int64_t(n), d); });
    for (size_t s = 0; s < n; ++s) T[size_t(k)][s] = R(I.T[s]);
    st[size_t(k)] = BatchStatic{me->geo.data(), I.h.geo32.data(), me->unique_map.data(), I.h.owner_mp.data(),
                                I.h.chunks.data(), &status[size_t(k)], me->N, int(me->npm), d, 0};
    const double h = I.dt / I.n_sub;
    StepConsts<R> K{R(h), R(0.5 * h), R(h / 6.0), R(I.dt), R(1.0 / me->M), R(me->N), {0, 0, 0}, {0, 0, 0}};
    for (int r = 0; r < 3; ++r) {
      K.lo[r] = R(me->lo[r]);
      K.hi[r] = R(me->hi[r]);
    }
    B->call[k] = BatchCall<R>{I.steady ? un[size_t(k)].data() : uo[size_t(k)].data(), un[size_t(k)].data(),
                              T[size_t(k)].data(), Tn[size_t(k)].data(), I.n_sub, I.steady, K};
    const int64_t nc = int64_t(I.h.chunks.size());
    for (int64_t c = 0; c < nc; c += chunks_per_item)
      items.push_back(make_int4(k, int(c), int(nc - c < chunks_per_item ? nc - c : chunks_per_item), 0));
  }
  int counter = 0;
  B->inst = st.data();
  B->items = items.data();
  B->n_items = int(items.size());
  B->count = count;
  B->counter = &counter;
  host_launch(blocks, kAdvectThreads, [&] { k_advect_batch<R, 2, 8>(*B); });
  // every instance's interface copies: (instance, copy slot, owner slot)
  std::vector<int4> ghosts;
  for (int k = 0; k < count; ++k)
    for (const int2& g : inst[size_t(k)].h.ghosts) ghosts.push_back(make_int4(k, g.x, g.y, 0));
  const int ng = int(ghosts.size());
  if (ng > 0) host_launch(unsigned((ng + 255) / 256), 256, [&] { k_batch_ghost_copy<R>(*B, ghosts.data(), ng); });
  out.clear();
  int flags = 0;
  for (int k = 0; k < count; ++k) {
    out.insert(out.end(), Tn[size_t(k)].begin(), Tn[size_t(k)].end());
    flags |= int(status[size_t(k)]);
  }
  // every instance's result in node order: the owner copies, by k_gather
  for (int k = 0; k < count; ++k) {
    const elm_mesh_s* me = inst[size_t(k)].me;
    const int64_t nu = me->n_unique;
    std::vector<R> Tu(static_cast<size_t>(nu), R(0));
    host_launch(unsigned((nu + 255) / 256), 256,
                [&] { k_gather<R>(Tn[size_t(k)].data(), Tu.data(), me->owner.data(), nu, 1); });
    out.insert(out.end(), Tu.begin(), Tu.end());
  }
  return flags;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 1;
  std::vector<int64_t> hd;
  if (!read_n(f, hd, 4)) return 1;
  const int count = int(hd[0]), precision = int(hd[1]), cpi = int(hd[2]);
  const unsigned blocks = unsigned(hd[3]);
  if (count < 1 || count > kMaxBatch || cpi < 1 || blocks < 1) return 1;
  std::vector<Instance> inst(static_cast<size_t>(count));
  for (Instance& I : inst) {
    std::vector<int64_t> ih, Mc;
    std::vector<double> dtv, V;
    if (!read_n(f, ih, 6) || !read_n(f, dtv, 1)) return 1;
    const int dim = int(ih[0]);
    if (!read_n(f, V, size_t(ih[1] * dim)) || !read_n(f, Mc, size_t(ih[2] * (dim + 1)))) return 1;
    elm_mesh m = nullptr;
    if (elm_mesh_create(dim, ih[1], V.data(), ih[2], Mc.data(), int(ih[3]),
                        (precision == 0 ? ELM_FP64 : ELM_FP32) | ELM_HOST_ONLY, &m) != ELM_OK) {
      std::fprintf(stderr, "mesh: %s\n", elm_last_error());
      return 1;
    }
    I.me = m;
    I.steady = int(ih[4]);
    I.n_sub = int(ih[5]);
    I.dt = dtv[0];
    const size_t n = size_t(m->n_storage);
    if (!read_n(f, I.uo, n * dim) || !read_n(f, I.un, n * dim) || !read_n(f, I.T, n)) return 1;
    I.h = host_tables(m);
  }
  std::fclose(f);
  std::vector<double> out;
  const int flags = precision == 0 ? run<double>(inst, cpi, blocks, out) : run<float>(inst, cpi, blocks, out);
  for (Instance& I : inst) elm_mesh_destroy(I.me);
  FILE* g = std::fopen(argv[2], "wb");
  if (!g || std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 1;
  std::fclose(g);
  if (flags != 0) {
    std::fprintf(stderr, "status flags %d\n", flags);
    return 2;
  }
  return 0;
}
