// cg_host_kernels.cpp -- the diffusion solve's vector kernels (csrc/
// diffusion.cu: k_cg_start, k_cg_begin, k_cg_update with the last block's
// completion, k_cg_direction, k_norm2, k_sum_into, k_invert_diag,
// k_set_boundary, k_residual_to_float, k_add_correction, k_copy) compiled with g++ and
// run on the CPU, each block's threads together (CUDA_HOST_THREADS), under
// AddressSanitizer / UndefinedBehaviorSanitizer or ThreadSanitizer, in the
// order one CG iteration uses them, for a check of each kernel's effect
// against NumPy (tests/test_kernel_host.py).  No GPU.
//
// Input file (little-endian): int64 [n, precision (0: FP64, 1: FP32),
// blocks, budget], doubles [alpha, stop_rr], then [n] each: r, dinv, q, x, v
// (doubles) and bnd, act (uint8).  Output file (doubles): after k_cg_start r,
// z, p; the scalars after k_cg_begin (rz, rr, done); after k_cg_update (with
// the given alpha and q) x, r, z and the scalars (rz_new, rr, beta, iters,
// done); p after k_cg_direction; |r|^2 over act (k_norm2 + k_sum_into);
// k_invert_diag of v; k_set_boundary(x, v); k_residual_to_float of x (r32,
// d32); x + double(r32) (k_add_correction); a copy of k_set_boundary's
// result (k_copy).
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

template <class R>
std::vector<double> run(int64_t n, unsigned blocks, int budget, double alpha, double stop_rr,
                        const std::vector<double>* in, const std::vector<uint8_t>& bnd,
                        const std::vector<uint8_t>& act) {
  const size_t ns = static_cast<size_t>(n);
  std::vector<R> r(in[0].begin(), in[0].end()), dinv(in[1].begin(), in[1].end()), q(ns, R(0)),
      x(in[3].begin(), in[3].end()), v(in[4].begin(), in[4].end()), z(ns, R(0)), p(ns, R(0));
  std::vector<double> part(2 * size_t(blocks), 0.0), out;
  auto put = [&](const std::vector<R>& a) { out.insert(out.end(), a.begin(), a.end()); };
  Scalars sc{};
  host_launch(blocks, kRedThreads,
              [&] { k_cg_start<R>(r.data(), z.data(), p.data(), q.data(), dinv.data(), bnd.data(), act.data(), n, part.data()); });
  put(r);
  put(z);
  put(p);
  host_launch(1, kRedThreads, [&] { k_cg_begin(part.data(), int(blocks), &sc, stop_rr, budget); });
  out.push_back(sc.rz);
  out.push_back(sc.rr);
  out.push_back(sc.done);
  // the operator pass would set q and alpha
  q.assign(in[2].begin(), in[2].end());
  sc.alpha = alpha;
  sc.done = 0;
  host_launch(blocks, kRedThreads, [&] {
    k_cg_update<R>(x.data(), r.data(), z.data(), p.data(), q.data(), dinv.data(), act.data(), &sc, n, part.data());
  });
  put(x);
  put(r);
  put(z);
  out.push_back(sc.rz_new);
  out.push_back(sc.rr);
  out.push_back(sc.beta);
  out.push_back(sc.iters);
  out.push_back(sc.done);
  host_launch(blocks, kRedThreads, [&] { k_cg_direction<R>(p.data(), z.data(), &sc, n); });
  put(p);
  double nrm = 0.0;
  host_launch(blocks, kRedThreads, [&] { k_norm2<R>(r.data(), act.data(), n, part.data()); });
  host_launch(1, kRedThreads, [&] { k_sum_into(part.data(), int(blocks), &nrm); });
  out.push_back(nrm);
  const unsigned eb = unsigned((n + 255) / 256);
  std::vector<R> d(v);
  host_launch(eb, 256, [&] { k_invert_diag<R>(d.data(), bnd.data(), n); });
  put(d);
  std::vector<R> xb(x);
  host_launch(eb, 256, [&] { k_set_boundary<R>(xb.data(), v.data(), bnd.data(), n); });
  put(xb);
  std::vector<double> x64(xb.begin(), xb.end());
  std::vector<float> r32(ns), d32(ns, 1.0f);
  host_launch(eb, 256, [&] { k_residual_to_float(x64.data(), r32.data(), d32.data(), bnd.data(), n); });
  out.insert(out.end(), r32.begin(), r32.end());
  out.insert(out.end(), d32.begin(), d32.end());
  host_launch(eb, 256, [&] { k_add_correction(x64.data(), r32.data(), n); });
  out.insert(out.end(), x64.begin(), x64.end());
  std::vector<R> cp(ns, R(0));
  host_launch(eb, 256, [&] { k_copy<R>(cp.data(), xb.data(), n); });
  put(cp);
  return out;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 1;
  std::vector<int64_t> hd;
  std::vector<double> sc;
  if (!read_n(f, hd, 4) || !read_n(f, sc, 2)) return 1;
  const int64_t n = hd[0];
  std::vector<double> in[5];
  std::vector<uint8_t> bnd, act;
  for (auto& a : in)
    if (!read_n(f, a, size_t(n))) return 1;
  if (!read_n(f, bnd, size_t(n)) || !read_n(f, act, size_t(n))) return 1;
  std::fclose(f);
  const unsigned blocks = unsigned(hd[2]);
  const std::vector<double> out = hd[1] == 0 ? run<double>(n, blocks, int(hd[3]), sc[0], sc[1], in, bnd, act)
                                             : run<float>(n, blocks, int(hd[3]), sc[0], sc[1], in, bnd, act);
  FILE* g = std::fopen(argv[2], "wb");
  if (!g || std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 1;
  std::fclose(g);
  return 0;
}
