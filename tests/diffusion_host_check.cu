// diffusion_host_check.cu -- CPU check of the host-built structures of the
// diffusion operator (diffusion.cu): the per-class stencil weights of the
// macro interiors, the interior node lists and their warp items, and the
// assembled rows of the shared-face nodes.  For a random field x it forms
// scale (M + alpha A) x twice: directly, by adding every inside micro
// simplex's element matrices, and the way the kernels do (stencil rows over
// the interior lists, assembled face rows), and checks that every node off
// the Dirichlet boundary is covered exactly once, that no stencil neighbour
// leaves its macro, and that the two agree to rounding.  Host-only meshes;
// no GPU.  Built and run by tests/test_diffusion_host.py.
#include "diffusion.cu"
#include <cstdio>
#include <random>

using namespace elm;

static int check(int dim, int order, int level, const std::vector<double>& V, const std::vector<int64_t>& T) {
  elm_mesh m = nullptr;
  const int prec = ELM_FP64 | ELM_HOST_ONLY | (order == 1 ? ELM_P1 : 0);
  if (elm_mesh_create(dim, int64_t(V.size() / dim), V.data(), int64_t(T.size() / (dim + 1)), T.data(), level, prec, &m) != ELM_OK) {
    printf("create failed: %s\n", elm_last_error());
    return 1;
  }
  elm_mesh_s* me = m;
  DiffusionHost h = diffusion_host(me);
  const int d = me->dim, P = me->order, nb = n_local(d, P), np = n_perm(d), N = me->N, M = me->M;
  const size_t tab = size_t(nb) * nb * (1 + np);
  const double alpha = 0.37, scale = 1.3;
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1, 1);
  std::vector<double> xu(me->n_unique), xs(me->n_storage);
  for (auto& v : xu) v = U(rng);
  for (int64_t s = 0; s < me->n_storage; ++s) xs[s] = xu[me->unique_map[s]];
  // reference: assembled (M + alpha A) x per unique node, over every inside simplex
  std::vector<double> yref(me->n_unique, 0.0);
  for (int64_t mm = 0; mm < me->n_macros; ++mm) {
    const double* Mt = h.t64.data() + mm * tab;
    const double* At = Mt + size_t(nb) * nb;
    for (int c0 = 0; c0 < N; ++c0)
      for (int c1 = 0; c1 <= c0; ++c1)
        for (int c2 = 0; c2 <= (d == 3 ? c1 : 0); ++c2) {
          const int c[3] = {c0, c1, c2};
          for (int sg = 0; sg < np; ++sg) {
            int s3[3] = {0, 1, 2};
            perm_of(d, sg, s3);
            bool inside = true;
            for (int a = 0; a < d; ++a)
              for (int b = a + 1; b < d; ++b)
                if (c[s3[a]] == c[s3[b]] && s3[a] > s3[b]) inside = false;
            if (!inside) continue;
            int64_t u[10];
            for (int j = 0; j < nb; ++j) {
              int q[3] = {0, 0, 0};
              for (int r = 0; r < d; ++r) q[r] = P * c[r] + node_off(d, sg, j, r, P);
              const int64_t sl = mm * me->npm + (d == 3 ? int64_t(q[0]) * (q[0] + 1) * (q[0] + 2) / 6 + int64_t(q[1]) * (q[1] + 1) / 2 + q[2]
                                                        : int64_t(q[0]) * (q[0] + 1) / 2 + q[1]);
              u[j] = me->unique_map[sl];
            }
            for (int i = 0; i < nb; ++i)
              for (int j = 0; j < nb; ++j)
                yref[u[i]] += scale * (Mt[i * nb + j] + alpha * At[(size_t(sg) * nb + i) * nb + j]) * xu[u[j]];
          }
        }
  }
  double ymax = 0;
  for (double v : yref) ymax = std::max(ymax, std::fabs(v));
  std::vector<int> seen(me->n_unique, 0);
  double err = 0;
  // stencil pass (host emulation of k_stencil)
  const int nt = stencil_entries(d, P);
  auto tri2 = [](int k) { return k * (k + 1) / 2; };
  auto tri3 = [](int k) { return k * (k + 1) * (k + 2) / 6; };
  for (size_t it = 0; it < h.items.size(); ++it) {
    const int4 w = h.items[it];
    if (h.items[it / 4 * 4].x != w.x) { printf("group macro mismatch\n"); return 1; }
    for (int lane = 0; lane < w.w; ++lane) {
      const uint32_t pk = h.nodes[w.z + lane];
      const int q0 = d == 3 ? int(pk & 1023u) : int(pk & 0xFFFFu);
      const int q1 = d == 3 ? int((pk >> 10) & 1023u) : int(pk >> 16);
      const int q2 = d == 3 ? int(pk >> 20) : 0;
      const int64_t slot = int64_t(w.x) * me->npm + (d == 3 ? tri3(q0) + tri2(q1) + q2 : tri2(q0) + q1);
      const double* W = h.w64.data() + size_t(2) * nt * w.x;
      double v = 0;
      auto row = [&](auto S) {
        const int k = w.y;
        for (int e = 0; e < S.n[k]; ++e) {
          const int* o = S.off[k][e];
          const int64_t nsl = d == 3 ? slot + (tri3(q0 + o[0]) - tri3(q0)) + (tri2(q1 + o[1]) - tri2(q1)) + o[2]
                                     : slot + (tri2(q0 + o[0]) - tri2(q0)) + o[1];
          if (nsl < w.x * me->npm || nsl >= (w.x + 1) * me->npm) { printf("neighbour outside the macro\n"); exit(1); }
          v += scale * (W[S.start[k] + e] + alpha * W[nt + S.start[k] + e]) * xs[nsl];
        }
      };
      if (d == 3 && P == 2) row(StencilShape<3, 2>{});
      else if (d == 3) row(StencilShape<3, 1>{});
      else if (P == 2) row(StencilShape<2, 2>{});
      else row(StencilShape<2, 1>{});
      const int64_t u = me->unique_map[slot];
      seen[u] += 1;
      err = std::max(err, std::fabs(v - yref[u]));
    }
  }
  // face rows
  const RowsHost& R = h.rows;
  for (size_t r = 0; r + 1 < R.off.size(); ++r) {
    double v = 0;
    for (int e = R.off[r]; e < R.off[r + 1]; ++e) v += scale * (R.wm[e] + alpha * R.wa[e]) * xs[R.col[e]];
    const int64_t u = me->unique_map[R.copies[R.copy_off[r]]];
    if (me->owner[u] != R.copies[R.copy_off[r]]) { printf("row's first copy is not the owner\n"); return 1; }
    seen[u] += 1;
    err = std::max(err, std::fabs(v - yref[u]));
  }
  int64_t bad = 0, nb_ = 0;
  for (int64_t u = 0; u < me->n_unique; ++u) {
    if (h.dbnd[u]) { nb_++; if (seen[u] != 0) bad++; }
    else if (seen[u] != 1) bad++;
  }
  printf("dim %d P%d level %d: unique %lld, boundary %lld, interior-list %zu, face rows %zu (nnz %zu), coverage errors %lld, max |dy| %.3e of %.3e\n",
         dim, order, level, (long long)me->n_unique, (long long)nb_, h.nodes.size(), R.off.size() - 1, R.col.size(),
         (long long)bad, err, ymax);
  elm_mesh_destroy(m);
  return (bad == 0 && err <= 1e-12 * ymax) ? 0 : 1;
}

int main() {
  std::vector<double> cube = {0,0,0, 1,0,0, 0,1,0, 1,1,0, 0,0,1, 1,0,1, 0,1,1, 1,1,1};
  std::vector<int64_t> ct = {0,1,3,7, 0,1,5,7, 0,2,3,7, 0,2,6,7, 0,4,5,7, 0,4,6,7};
  std::vector<double> sq = {0,0, 1,0, 0,1, 1,1};
  std::vector<int64_t> st = {0,1,3, 0,2,3};
  // a perturbed 2 x 2 x 2 block of cubes (48 macros)
  std::vector<double> bv;
  std::vector<int64_t> bt;
  std::mt19937_64 g(3);
  std::uniform_real_distribution<double> U(-0.08, 0.08);
  for (int k = 0; k < 3; ++k) for (int j = 0; j < 3; ++j) for (int i = 0; i < 3; ++i) {
    const bool in = i == 1 && j == 1 && k == 1;
    bv.push_back(i * 0.5 + (in ? U(g) : 0)); bv.push_back(j * 0.5 + (in ? U(g) : 0)); bv.push_back(k * 0.5 + (in ? U(g) : 0));
  }
  for (int k = 0; k < 2; ++k) for (int j = 0; j < 2; ++j) for (int i = 0; i < 2; ++i) {
    auto id = [&](int a, int b, int c) { return int64_t((k + c) * 9 + (j + b) * 3 + (i + a)); };
    const int64_t c0 = id(0,0,0), c7 = id(1,1,1);
    const int64_t e[3] = {id(1,0,0), id(0,1,0), id(0,0,1)};
    const int perms[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
    for (auto& p : perms) {
      int a[3] = {0,0,0}; a[p[0]] = 1; const int64_t v1 = id(a[0], a[1], a[2]);
      a[p[1]] = 1; const int64_t v2 = id(a[0], a[1], a[2]);
      (void)e;
      bt.push_back(c0); bt.push_back(v1); bt.push_back(v2); bt.push_back(c7);
    }
  }
  int rc = 0;
  for (int lv : {0, 1, 2, 3, 4}) {
    rc |= check(3, 2, lv, cube, ct);
    rc |= check(3, 1, lv, cube, ct);
    rc |= check(2, 2, lv, sq, st);
    rc |= check(2, 1, lv, sq, st);
  }
  rc |= check(3, 2, 2, bv, bt);
  rc |= check(3, 1, 3, bv, bt);
  printf(rc ? "FAILED\n" : "all ok\n");
  return rc;
}
