// adjoint_host_check.cpp -- the adjoint's device code (csrc/adjoint_kernels.cuh)
// compiled with g++ and run on the CPU for a CPU parity check against the
// oracle's transpose and forward-mode derivative (tests/test_kernel_host.py),
// under AddressSanitizer and UndefinedBehaviorSanitizer.  No GPU.
//
// It replays launch_adjoint's sequence on the host, one thread at a time:
// pass 0 of k_adjoint over the work list, the interface copies' statistics
// merged into their owners, the scale exponents, the owners' exponents handed
// back to the copies, pass 1, the copies' sums folded into their owners, and
// the scaling back.
//
// Input file (little-endian): int64 header [dim, n_vertices, n_macros, level,
// precision (0: FP64, 1: FP32), order, steady, n_sub, split], double dt, vertex
// coordinates, macro vertices (int64; 2D or 3D), then in the storage layout u^n, u^{n+1}
// [n_storage * dim], T^n [n_storage] and the incoming gradient dL/dT^{n+1}
// [n_storage] (doubles).  split = 1 keeps the gradients of u^n and u^{n+1}
// apart (time-dependent velocity).  Output file: dL/dT^n [n_storage], dL/du^n
// and dL/du^{n+1} [n_storage * dim] each (doubles; copies of interface nodes
// hold 0, their owner the sum).  Exit status: 0, 1 on bad input, 2 on a
// device-side status flag.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "adjoint_kernels.cuh"
#include "host_mesh_tables.h"

using namespace elm;
using elm_host_check::HostTables;
using elm_host_check::host_tables;

namespace {

// A one-dimensional launch of `count` threads in blocks of 256, one thread
// at a time.
template <class F>
void grid1d(int64_t count, F kernel) {
  blockDim.x = 256;
  const int64_t blocks = (count + 255) / 256;
  for (int64_t b = 0; b < blocks; ++b) {
    blockIdx.x = unsigned(b);
    for (unsigned t = 0; t < 256; ++t) {
      threadIdx.x = t;
      kernel();
    }
  }
}

template <int D, class R, bool STEADY, int P>
unsigned adjoint(elm_mesh_s* me, const HostTables& h, bool split, const std::vector<double>& uo_in,
                 const std::vector<double>& un_in, const std::vector<double>& T_in,
                 const std::vector<double>& g_in, double dt, int n_sub, std::vector<double>& out) {
  const int64_t n = me->n_storage;
  const size_t ns = static_cast<size_t>(n);
  std::vector<R> un(ns * 4, R(0)), uo(ns * 4, R(0)), T(ns, R(0)), g(ns, R(0));
  for (size_t s = 0; s < ns; ++s) {
    for (int r = 0; r < D; ++r) {
      un[s * 4 + r] = R(un_in[s * D + r]);
      uo[s * 4 + r] = R(uo_in[s * D + r]);
    }
    T[s] = R(T_in[s]);
    g[s] = R(g_in[s]);
  }
  unsigned status = 0;
  const double hstep = dt / n_sub;
  AdvectArgs a{};
  a.geo = me->geo.data();
  a.geo32 = h.geo32.data();
  a.n_macros = int32_t(me->n_macros);
  a.N = me->N;
  a.npm = me->npm;
  a.n_storage = n;
  for (int r = 0; r < 3; ++r) {
    a.lo[r] = me->lo[r];
    a.hi[r] = me->hi[r];
  }
  a.u_new = un.data();
  a.u_old = STEADY ? un.data() : uo.data();
  a.steady = STEADY;
  a.T_old = T.data();
  a.dt = dt;
  a.n_sub = n_sub;
  a.status = &status;
  a.unique_map = me->unique_map.data();
  a.owner_mp = h.owner_mp.data();
  a.chunks = h.chunks.data();
  a.n_chunks = int(h.chunks.size());
  a.ghosts = h.ghosts.data();
  a.n_ghosts = int(h.ghosts.size());
  a.skip_ghosts = 1;
  a.order = me->order;
  a.k64 = {hstep, 0.5 * hstep, hstep / 6.0, dt, 1.0 / me->M, double(me->N), {0, 0, 0}, {0, 0, 0}};
  a.k32 = {float(hstep), float(0.5 * hstep), float(hstep / 6.0), float(dt), float(1.0 / me->M), float(me->N),
           {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < 3; ++r) {
    a.k64.lo[r] = me->lo[r];
    a.k64.hi[r] = me->hi[r];
    a.k32.lo[r] = float(me->lo[r]);
    a.k32.hi[r] = float(me->hi[r]);
  }
  const int nsets = (!STEADY && split) ? 2 : 1;
  const int64_t nstat = n * (1 + nsets);
  std::vector<unsigned long long> acc_T(ns, 0ull), acc_U(ns * D * 2, 0ull), smax(ns * 3, 0ull), scnt(ns * 3, 0ull);
  std::vector<int> kexp(ns * 3, 0);
  AdjArgs aa{g.data(), acc_T.data(), acc_U.data(), smax.data(), scnt.data(), kexp.data(), nsets == 2 ? 1 : 0, 0};
  Tables<R> tab;
  if constexpr (sizeof(R) == 8)
    tab.g = me->geo.data();
  else
    tab.g = h.geo32.data();
  const int ng = int(h.ghosts.size());
  for (int pass = 0; pass < 2; ++pass) {
    aa.pass = pass;
    blockDim.x = kAdvectThreads;
    for (int b = 0; b < a.n_chunks; ++b) {
      blockIdx.x = unsigned(b);
      for (unsigned t = 0; t < unsigned(kAdvectThreads); ++t) {
        threadIdx.x = t;
        if (pass == 0)
          k_adjoint<D, R, STEADY, P, 0>(a, aa, tab, 0);
        else
          k_adjoint<D, R, STEADY, P, 1>(a, aa, tab, 0);
      }
    }
    if (pass == 0) {
      if (ng > 0)
        grid1d(int64_t(ng) * (1 + nsets),
               [&] { k_merge_stats(smax.data(), scnt.data(), n, 1 + nsets, h.ghosts.data(), ng); });
      grid1d(nstat, [&] { k_scales<R>(smax.data(), scnt.data(), kexp.data(), nstat, &status); });
      if (ng > 0) grid1d(int64_t(ng) * (1 + nsets), [&] { k_copy_scales(kexp.data(), n, 1 + nsets, h.ghosts.data(), ng); });
    }
  }
  grid1d(n, [&] { k_fold_ghosts(acc_T.data(), 1, 1, n, me->unique_map.data(), me->owner.data()); });
  grid1d(n, [&] { k_fold_ghosts(acc_U.data(), D, nsets, n, me->unique_map.data(), me->owner.data()); });
  std::vector<R> gT(ns, R(0)), gU0(ns * D, R(0)), gU1(ns * D, R(0));
  grid1d(n, [&] { k_scale_out<R>(acc_T.data(), gT.data(), n, 1, kexp.data()); });
  grid1d(n * D, [&] { k_scale_out<R>(acc_U.data(), gU0.data(), n, D, kexp.data() + n); });
  if (nsets == 2) grid1d(n * D, [&] { k_scale_out<R>(acc_U.data() + n * D, gU1.data(), n, D, kexp.data() + 2 * n); });
  out.clear();
  out.insert(out.end(), gT.begin(), gT.end());
  out.insert(out.end(), gU0.begin(), gU0.end());
  out.insert(out.end(), gU1.begin(), gU1.end());
  return status;
}

template <int D, class R>
unsigned dispatch(elm_mesh_s* me, const HostTables& h, bool steady, bool split, const std::vector<double>& uo,
                  const std::vector<double>& un, const std::vector<double>& T, const std::vector<double>& g,
                  double dt, int n_sub, std::vector<double>& out) {
  if (me->order == 1)
    return steady ? adjoint<D, R, true, 1>(me, h, split, uo, un, T, g, dt, n_sub, out)
                  : adjoint<D, R, false, 1>(me, h, split, uo, un, T, g, dt, n_sub, out);
  return steady ? adjoint<D, R, true, 2>(me, h, split, uo, un, T, g, dt, n_sub, out)
                : adjoint<D, R, false, 2>(me, h, split, uo, un, T, g, dt, n_sub, out);
}

template <class T>
bool read_n(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s input output\n", argv[0]);
    return 1;
  }
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 1;
  std::vector<int64_t> hd;
  std::vector<double> dtv;
  if (!read_n(f, hd, 9) || !read_n(f, dtv, 1)) return 1;
  const int dim = int(hd[0]), precision = int(hd[4]), order = int(hd[5]), n_sub = int(hd[7]);
  const bool steady = hd[6] != 0, split = hd[8] != 0;
  std::vector<double> V;
  std::vector<int64_t> Mc;
  if (!read_n(f, V, size_t(hd[1] * dim)) || !read_n(f, Mc, size_t(hd[2] * (dim + 1)))) return 1;
  elm_mesh mesh = nullptr;
  const int prec = (precision == 0 ? ELM_FP64 : ELM_FP32) | ELM_HOST_ONLY | (order == 1 ? ELM_P1 : 0);
  if (elm_mesh_create(dim, hd[1], V.data(), hd[2], Mc.data(), int(hd[3]), prec, &mesh) != ELM_OK) {
    std::fprintf(stderr, "mesh: %s\n", elm_last_error());
    return 1;
  }
  const int64_t n = mesh->n_storage;
  std::vector<double> uo, un, T, g, out;
  if (!read_n(f, uo, size_t(n * dim)) || !read_n(f, un, size_t(n * dim)) || !read_n(f, T, size_t(n)) ||
      !read_n(f, g, size_t(n)))
    return 1;
  std::fclose(f);
  const HostTables h = host_tables(mesh);
  unsigned status;
  if (dim == 3)
    status = precision == 0 ? dispatch<3, double>(mesh, h, steady, split, uo, un, T, g, dtv[0], n_sub, out)
                            : dispatch<3, float>(mesh, h, steady, split, uo, un, T, g, dtv[0], n_sub, out);
  else
    status = precision == 0 ? dispatch<2, double>(mesh, h, steady, split, uo, un, T, g, dtv[0], n_sub, out)
                            : dispatch<2, float>(mesh, h, steady, split, uo, un, T, g, dtv[0], n_sub, out);
  elm_mesh_destroy(mesh);
  FILE* o = std::fopen(argv[2], "wb");
  if (!o || std::fwrite(out.data(), sizeof(double), out.size(), o) != out.size()) return 1;
  std::fclose(o);
  if (status != 0) {
    std::fprintf(stderr, "status flags %u\n", status);
    return 2;
  }
  return 0;
}
