// diffusion_host_kernels.cpp -- the diffusion operator's kernels (k_stencil over
// the macro interiors, k_face_rows over the nodes of shared faces; csrc/
// diffusion.cu) compiled with g++ and run on the CPU, each block's threads
// together (CUDA_HOST_THREADS in tests/cuda_host_shim.h: barriers, warp
// shuffles), under AddressSanitizer and UndefinedBehaviorSanitizer, for a CPU
// check against the oracle's assembled matrices (tests/test_kernel_host.py).
// No GPU.
//
// The test writes diffusion_front.cuh: the part of diffusion.cu before the
// device set-up (kernels and host-built structures, no launches).  The
// structures come from diffusion_host(); the operator pass accumulates
// y = scale (M + alpha A) x over the interior nodes (stencils) and the rows of
// the shared-face nodes, as apply_op launches them (kOpAccum, y starting at
// 0).  Dirichlet nodes get no row.  With cg = 1 the passes run as in a CG
// iteration (kOpCg): y = v, one partial of p.q per block, and the last block
// of the face-row pass (or of the stencil pass, without face rows) sums all
// partials in a fixed order into the scalars (p = x).  With cg = 2 they add
// the diagonal entry of each row instead (kOpDiag, x unused), as the Jacobi
// preconditioner's set-up runs them.
//
// Input file (little-endian): int64 header [dim, n_vertices, n_macros, level,
// precision (0: FP64, 1: FP32), order, cg (0, 1 or 2)], doubles [alpha, scale], vertex
// coordinates, macro vertices (int64), x [n_storage] (doubles).  Output file:
// y [n_storage], then p.q (doubles).  Exit status 0, or 1 on bad input.
#include <cstdio>
#include <vector>

#include "diffusion_front.cuh"

using namespace elm;

namespace {

template <class T>
bool read_n(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

template <int D, class R, int P, int MODE>
void apply(elm_mesh_s* me, const std::vector<double>& x_in, double alpha, double scale, std::vector<double>& out) {
  const DiffusionHost h = diffusion_host(me);
  const size_t n = size_t(me->n_storage);
  std::vector<R> x(n), y(n, R(0));
  for (size_t s = 0; s < n; ++s) x[s] = R(x_in[s]);
  std::vector<R> w(h.w64.begin(), h.w64.end());
  StencilArgs st{};
  st.wtab = w.data();
  st.nodes = h.nodes.data();
  st.items = h.items.data();
  st.n_groups = int64_t(h.items.size() / 4);
  st.npm = int(me->npm);
  const unsigned nsb = unsigned(st.n_groups < 6 ? st.n_groups : 6);  // persistent over the groups
  const int64_t n_rows = int64_t(h.rows.off.size()) - 1;
  const unsigned nfb = unsigned(n_rows == 0 ? 0 : n_rows < 24 ? (n_rows + 7) / 8 : 3);  // 8 rows (warps) per block
  Scalars sc{};
  sc.rz = 1.0;
  sc.budget = 1 << 30;
  std::vector<double> part(nsb + nfb + 1, 0.0);
  const bool cg = MODE == kOpCg;
  st.sc = cg ? &sc : nullptr;
  st.finish = cg && nfb == 0 ? int(nsb) : 0;
  if (nsb > 0)
    host_launch(nsb, 128, [&] { k_stencil<D, R, P, MODE>(st, x.data(), y.data(), R(alpha), R(scale), part.data()); });
  std::vector<R> fw(h.rows.wm.begin(), h.rows.wm.end());
  fw.insert(fw.end(), h.rows.wa.begin(), h.rows.wa.end());
  FaceRows fr{};
  fr.off = h.rows.off.data();
  fr.col = h.rows.col.data();
  fr.w = fw.data();
  fr.nnz = int64_t(h.rows.wm.size());
  fr.copy_off = h.rows.copy_off.data();
  fr.copies = h.rows.copies.data();
  fr.n = n_rows;
  fr.sc = cg ? &sc : nullptr;
  fr.finish = cg ? int(nsb + nfb) : 0;
  fr.part0 = part.data();
  if (nfb > 0)
    host_launch(nfb, kRedThreads,
                [&] { k_face_rows<R, MODE>(fr, x.data(), y.data(), R(alpha), R(scale), part.data() + nsb); });
  out.assign(y.begin(), y.end());
  out.push_back(sc.pq);
}

template <int MODE>
void dispatch(elm_mesh_s* me, int dim, int precision, int order, const std::vector<double>& x, double alpha,
              double scale, std::vector<double>& out) {
  if (dim == 3) {
    if (precision == 0)
      order == 2 ? apply<3, double, 2, MODE>(me, x, alpha, scale, out) : apply<3, double, 1, MODE>(me, x, alpha, scale, out);
    else
      order == 2 ? apply<3, float, 2, MODE>(me, x, alpha, scale, out) : apply<3, float, 1, MODE>(me, x, alpha, scale, out);
  } else {
    if (precision == 0)
      order == 2 ? apply<2, double, 2, MODE>(me, x, alpha, scale, out) : apply<2, double, 1, MODE>(me, x, alpha, scale, out);
    else
      order == 2 ? apply<2, float, 2, MODE>(me, x, alpha, scale, out) : apply<2, float, 1, MODE>(me, x, alpha, scale, out);
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 1;
  std::vector<int64_t> hd;
  std::vector<double> ab, V, x, out;
  std::vector<int64_t> Mc;
  if (!read_n(f, hd, 7) || !read_n(f, ab, 2)) return 1;
  const int dim = int(hd[0]), precision = int(hd[4]), order = int(hd[5]);
  const bool cg = hd[6] != 0;
  if (!read_n(f, V, size_t(hd[1] * dim)) || !read_n(f, Mc, size_t(hd[2] * (dim + 1)))) return 1;
  elm_mesh mesh = nullptr;
  const int prec = (precision == 0 ? ELM_FP64 : ELM_FP32) | ELM_HOST_ONLY | (order == 1 ? ELM_P1 : 0);
  if (elm_mesh_create(dim, hd[1], V.data(), hd[2], Mc.data(), int(hd[3]), prec, &mesh) != ELM_OK) {
    std::fprintf(stderr, "mesh: %s\n", elm_last_error());
    return 1;
  }
  if (!read_n(f, x, size_t(mesh->n_storage))) return 1;
  std::fclose(f);
  if (hd[6] == 2)
    dispatch<kOpDiag>(mesh, dim, precision, order, x, ab[0], ab[1], out);
  else if (cg)
    dispatch<kOpCg>(mesh, dim, precision, order, x, ab[0], ab[1], out);
  else
    dispatch<kOpAccum>(mesh, dim, precision, order, x, ab[0], ab[1], out);
  elm_mesh_destroy(mesh);
  FILE* g = std::fopen(argv[2], "wb");
  if (!g || std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 1;
  std::fclose(g);
  return 0;
}
