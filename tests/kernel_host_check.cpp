// kernel_host_check.cpp -- the advection step's kernels (csrc/advect.cu:
// k_pack_velocity, k_advect, k_ghost_copy; the per-node work in csrc/
// tracer.cuh) compiled with g++ and run on the CPU, one thread at a time, for
// a CPU parity check against the oracle (tests/test_kernel_host.py) under
// AddressSanitizer and UndefinedBehaviorSanitizer.  No GPU.
//
// The test writes advect_front.cuh, the part of advect.cu before its launch
// functions.  The program launches what elm_set_velocity and elm_advect
// launch, with the same arguments: the velocity records (k_pack_velocity), the
// per-node kernel over the host-built work list (kAdvectSplit blocks per chunk
// of up to 128 nodes of one slab of one macro; each interface node computed
// once, in its owner's slot) and the interface copies (k_ghost_copy).
//
// Three per-node modes, as the GPU path has: the step (T^{n+1} = T^n_h(X)),
// a trace over one interval (from the node, or continued from given offsets;
// the new offsets X - x_i are the result) and the evaluation of T at x_i plus
// given offsets.
//
// Input file (little-endian, as numpy writes it): int64 header [dim,
// n_vertices, n_macros, level, precision (0: FP64, 1: FP32), order, steady,
// n_sub, mode (0: step, 1: trace, 2: evaluation), offsets given (0 / 1)],
// doubles [dt, r_min, r_max, n_sectors, theta0] (n_sectors > 0: the mesh is
// blended onto that annulus; 2D FP64), vertex coordinates [n_vertices * dim], macro vertices
// [n_macros * (dim + 1)] (int64), then in the mesh's storage layout u^n and
// u^{n+1} [n_storage * dim], T^n [n_storage] and, if given, the offsets
// [n_storage * dim] (doubles, already rounded to FP32 for an FP32 run).
// Output file: T^{n+1} [n_storage] (step, evaluation) or the offsets
// [n_storage * dim] (trace), doubles.  Exit status: 0, 1 on bad input, 2 on a
// device-side status flag.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "advect_front.cuh"
#include "host_mesh_tables.h"

using namespace elm;
using elm_host_check::HostTables;
using elm_host_check::host_tables;
using elm_host_check::sector_table;

namespace {

template <class R>
StepConsts<R> step_consts(const elm_mesh_s* me, double dt, int n_sub) {
  const double h = dt / n_sub;
  StepConsts<R> K{R(h), R(0.5 * h), R(h / 6.0), R(dt), R(1.0 / me->M), R(me->N), {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < 3; ++r) {
    K.lo[r] = R(me->lo[r]);
    K.hi[r] = R(me->hi[r]);
  }
  return K;
}

template <int D, class R, bool STEADY, int P, int MODE, int BLEND>
unsigned step(const elm_mesh_s* me, const HostTables& h, const std::vector<double>& uo_in,
              const std::vector<double>& un_in, const std::vector<double>& T_in, const std::vector<double>* D_in,
              double dt, int n_sub, std::vector<double>& out) {
  const int64_t n = me->n_storage;
  const size_t ns = static_cast<size_t>(n);
  // velocity records by k_pack_velocity, as elm_set_velocity makes them
  std::vector<R> u_un(ns * D), u_uo(ns * D), un(ns * 4, R(0)), uo(ns * 4, R(0)), T(ns, R(0)), Tn(ns, R(0)), Din,
      Dout(ns * D, R(0));
  for (size_t s = 0; s < ns * D; ++s) {
    u_un[s] = R(un_in[s]);
    u_uo[s] = R(uo_in[s]);
  }
  const unsigned pb = unsigned((n + 255) / 256);
  host_serial_launch(pb, 256, [&] { k_pack_velocity<R>(u_un.data(), un.data(), n, D); });
  host_serial_launch(pb, 256, [&] { k_pack_velocity<R>(u_uo.data(), uo.data(), n, D); });
  for (size_t s = 0; s < ns; ++s) T[s] = R(T_in[s]);
  if (D_in) Din.assign(D_in->begin(), D_in->end());
  unsigned status = 0;
  // the launch arguments, as make_args builds them
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
  a.T_new = Tn.data();
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
  a.mode = MODE;
  a.D_in = D_in ? static_cast<const void*>(Din.data()) : nullptr;
  a.D_out = Dout.data();
  a.blend = me->blend;
  const double hs = dt / n_sub;
  a.k64 = {hs, 0.5 * hs, hs / 6.0, dt, 1.0 / me->M, double(me->N), {0, 0, 0}, {0, 0, 0}};
  a.k32 = {float(hs), float(0.5 * hs), float(hs / 6.0), float(dt), float(1.0 / me->M), float(me->N), {0, 0, 0},
           {0, 0, 0}};
  for (int r = 0; r < 3; ++r) {
    a.k64.lo[r] = me->lo[r];
    a.k64.hi[r] = me->hi[r];
    a.k32.lo[r] = float(me->lo[r]);
    a.k32.hi[r] = float(me->hi[r]);
  }
  Tables<R> tab;
  if constexpr (sizeof(R) == 8)
    tab.g = me->geo.data();
  else
    tab.g = h.geo32.data();
  // k_advect over the work list (kAdvectSplit blocks per chunk), then
  // k_ghost_copy for the interface copies
  host_serial_launch(unsigned(a.n_chunks) * kAdvectSplit, kStepThreads,
                     [&] { k_advect<D, R, STEADY, P, MODE, BLEND>(a, tab, 0); });
  const int ncomp = MODE == kTrace ? D : 1;
  R* res = MODE == kTrace ? Dout.data() : Tn.data();
  if (a.n_ghosts > 0)
    host_serial_launch(unsigned((int64_t(a.n_ghosts) * ncomp + 255) / 256), 256,
                       [&] { k_ghost_copy<R>(a.ghosts, a.n_ghosts, res, ncomp); });
  if (MODE == kTrace)
    out.assign(Dout.begin(), Dout.end());
  else
    out.assign(Tn.begin(), Tn.end());
  return status;
}

template <int D, class R, int MODE, int BLEND>
unsigned dispatch_blend(const elm_mesh_s* me, const HostTables& h, bool steady, const std::vector<double>& uo,
                        const std::vector<double>& un, const std::vector<double>& T, const std::vector<double>* Di,
                        double dt, int n_sub, std::vector<double>& out) {
  if (me->order == 1)
    return steady ? step<D, R, true, 1, MODE, BLEND>(me, h, uo, un, T, Di, dt, n_sub, out)
                  : step<D, R, false, 1, MODE, BLEND>(me, h, uo, un, T, Di, dt, n_sub, out);
  return steady ? step<D, R, true, 2, MODE, BLEND>(me, h, uo, un, T, Di, dt, n_sub, out)
                : step<D, R, false, 2, MODE, BLEND>(me, h, uo, un, T, Di, dt, n_sub, out);
}

template <int D, class R, int MODE>
unsigned dispatch_mode(const elm_mesh_s* me, const HostTables& h, bool steady, const std::vector<double>& uo,
                       const std::vector<double>& un, const std::vector<double>& T, const std::vector<double>* Di,
                       double dt, int n_sub, std::vector<double>& out) {
  if constexpr (D == 2 && sizeof(R) == 8) {
    if (me->blend.nsec > 0) return dispatch_blend<D, R, MODE, 1>(me, h, steady, uo, un, T, Di, dt, n_sub, out);
  }
  return dispatch_blend<D, R, MODE, 0>(me, h, steady, uo, un, T, Di, dt, n_sub, out);
}

template <int D, class R>
unsigned dispatch(const elm_mesh_s* me, const HostTables& h, int mode, bool steady, const std::vector<double>& uo,
                  const std::vector<double>& un, const std::vector<double>& T, const std::vector<double>* Di,
                  double dt, int n_sub, std::vector<double>& out) {
  if (mode == kTrace) return dispatch_mode<D, R, kTrace>(me, h, steady, uo, un, T, Di, dt, n_sub, out);
  if (mode == kEval) return dispatch_mode<D, R, kEval>(me, h, steady, uo, un, T, Di, dt, n_sub, out);
  return dispatch_mode<D, R, kStep>(me, h, steady, uo, un, T, Di, dt, n_sub, out);
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
  if (!read_n(f, hd, 10) || !read_n(f, dtv, 5)) return 1;
  const int dim = int(hd[0]), precision = int(hd[4]), order = int(hd[5]), n_sub = int(hd[7]), mode = int(hd[8]);
  const bool steady = hd[6] != 0, has_din = hd[9] != 0;
  if (mode < kStep || mode > kEval || (mode == kEval && !has_din)) return 1;
  std::vector<double> V;
  std::vector<int64_t> Mc;
  if (!read_n(f, V, size_t(hd[1] * dim)) || !read_n(f, Mc, size_t(hd[2] * (dim + 1)))) return 1;
  elm_mesh mesh = nullptr;
  const int prec = (precision == 0 ? ELM_FP64 : ELM_FP32) | ELM_HOST_ONLY | (order == 1 ? ELM_P1 : 0);
  if (elm_mesh_create(dim, hd[1], V.data(), hd[2], Mc.data(), int(hd[3]), prec, &mesh) != ELM_OK) {
    std::fprintf(stderr, "mesh: %s\n", elm_last_error());
    return 1;
  }
  std::vector<double> sec;
  if (dtv[3] > 0) {
    if (elm_mesh_set_annulus(mesh, dtv[1], dtv[2], int(dtv[3]), dtv[4]) != ELM_OK) {
      std::fprintf(stderr, "annulus: %s\n", elm_last_error());
      return 1;
    }
    sec = sector_table(int(dtv[3]), dtv[4]);  // a host-only mesh keeps no copy of it
    mesh->blend.sec = sec.data();
  }
  const int64_t n = mesh->n_storage;
  std::vector<double> uo, un, T, Di, out;
  if (!read_n(f, uo, size_t(n * dim)) || !read_n(f, un, size_t(n * dim)) || !read_n(f, T, size_t(n)) ||
      (has_din && !read_n(f, Di, size_t(n * dim))))
    return 1;
  const std::vector<double>* dptr = has_din ? &Di : nullptr;
  std::fclose(f);
  const HostTables h = host_tables(mesh);
  unsigned status;
  if (dim == 3)
    status = precision == 0 ? dispatch<3, double>(mesh, h, mode, steady, uo, un, T, dptr, dtv[0], n_sub, out)
                            : dispatch<3, float>(mesh, h, mode, steady, uo, un, T, dptr, dtv[0], n_sub, out);
  else
    status = precision == 0 ? dispatch<2, double>(mesh, h, mode, steady, uo, un, T, dptr, dtv[0], n_sub, out)
                            : dispatch<2, float>(mesh, h, mode, steady, uo, un, T, dptr, dtv[0], n_sub, out);
  mesh->blend.sec = nullptr;  // owned by `sec`
  elm_mesh_destroy(mesh);
  FILE* g = std::fopen(argv[2], "wb");
  if (!g || std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 1;
  std::fclose(g);
  if (status != 0) {
    std::fprintf(stderr, "status flags %u\n", status);
    return 2;
  }
  return 0;
}
