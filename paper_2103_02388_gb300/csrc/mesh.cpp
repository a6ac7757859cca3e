// mesh.cpp -- host construction of the block-structured P2 mesh (Sec. 2.1 and
// Sec. 2.3.1, grid data structure of arXiv 2103.02388): macro affine maps, face
// neighbours, storage layout and the owner of every interface node.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

#include "elm_internal.h"

namespace elm {
namespace {

bool invert(int d, const double* A, double* Ainv) {
  if (d == 2) {
    const double det = A[0] * A[3] - A[1] * A[2];
    if (det == 0.0 || !std::isfinite(det)) return false;
    Ainv[0] = A[3] / det;
    Ainv[1] = -A[1] / det;
    Ainv[2] = -A[2] / det;
    Ainv[3] = A[0] / det;
    return true;
  }
  const double c00 = A[4] * A[8] - A[5] * A[7];
  const double c01 = A[5] * A[6] - A[3] * A[8];
  const double c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (det == 0.0 || !std::isfinite(det)) return false;
  Ainv[0] = c00 / det;
  Ainv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ainv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ainv[3] = c01 / det;
  Ainv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ainv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ainv[6] = c02 / det;
  Ainv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ainv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return true;
}

// Key of an interface node: (vertex id, integer barycentric weight) pairs of
// the non-zero weights, in ascending vertex id.  Unused pairs are -1.
using NodeKey = std::array<int64_t, 8>;
struct NodeKeyHash {
  size_t operator()(const NodeKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : k) {
      h ^= uint64_t(v) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    }
    return size_t(h);
  }
};

}  // namespace

elm_status build_mesh(int dim, int64_t nv, const double* xyz, int64_t nm, const int64_t* mv,
                      int level, int precision, elm_mesh_s* me, std::string* err) {
  const int d = dim;
  me->dim = d;
  me->level = level;
  me->N = 1 << level;
  me->M = me->order * me->N;  // node lattice points per macro edge
  me->precision = precision;
  me->n_macros = nm;
  me->npm = nodes_per_macro(d, me->M);
  me->n_storage = nm * me->npm;
  for (int r = 0; r < 3; ++r) {
    me->lo[r] = 0.0;
    me->hi[r] = 0.0;
  }
  for (int r = 0; r < d; ++r) {
    me->lo[r] = HUGE_VAL;
    me->hi[r] = -HUGE_VAL;
  }
  for (int64_t i = 0; i < nv * d; ++i) {
    if (!std::isfinite(xyz[i])) {
      *err = "vertex coordinates must be finite";
      return ELM_ERR_ARG;
    }
    me->lo[i % d] = std::min(me->lo[i % d], xyz[i]);
    me->hi[i % d] = std::max(me->hi[i % d], xyz[i]);
  }

  // Macro affine maps with vertices in ascending id (Kuhn order).
  me->geo.assign(nm, MacroGeo{});
  std::vector<std::array<int64_t, 4>> verts(nm);
  for (int64_t m = 0; m < nm; ++m) {
    std::array<int64_t, 4> v{-1, -1, -1, -1};
    for (int k = 0; k <= d; ++k) {
      v[k] = mv[m * (d + 1) + k];
      if (v[k] < 0 || v[k] >= nv) {
        *err = "macro " + std::to_string(m) + ": vertex id out of range";
        return ELM_ERR_ARG;
      }
    }
    // ascending ids (at most 4: insertion sort)
    for (int i = 1; i <= d; ++i)
      for (int j = i; j > 0 && v[j - 1] > v[j]; --j) std::swap(v[j - 1], v[j]);
    for (int k = 0; k < d; ++k)
      if (v[k] == v[k + 1]) {
        *err = "macro " + std::to_string(m) + ": repeated vertex";
        return ELM_ERR_TOPOLOGY;
      }
    verts[m] = v;
    MacroGeo& g = me->geo[m];
    for (int r = 0; r < d; ++r) g.v0[r] = xyz[v[0] * d + r];
    double J[9] = {0}, Jinv[9] = {0};
    double scale = 0.0;
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        J[r * d + c] = xyz[v[c + 1] * d + r] - xyz[v[c] * d + r];
        scale = std::max(scale, std::fabs(J[r * d + c]));
      }
    const double det = d == 2 ? J[0] * J[3] - J[1] * J[2]
                              : J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                                    J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(std::fabs(det) > 1e-12 * std::pow(scale, d)) || !invert(d, J, Jinv)) {
      *err = "macro " + std::to_string(m) + ": degenerate simplex";
      return ELM_ERR_TOPOLOGY;
    }
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        g.J[r * 3 + c] = J[r * d + c];
        g.NJinv[r * 3 + c] = double(me->N) * Jinv[r * d + c];
      }
    for (int k = 0; k < 4; ++k) g.nb[k] = -1;
  }

  // Face neighbours: face k of macro m is opposite its local vertex k.
  std::map<std::array<int64_t, 3>, std::vector<std::pair<int64_t, int>>> faces;
  for (int64_t m = 0; m < nm; ++m)
    for (int k = 0; k <= d; ++k) {
      std::array<int64_t, 3> f{-1, -1, -1};
      int n = 0;
      for (int j = 0; j <= d; ++j)
        if (j != k) f[n++] = verts[m][j];
      faces[f].push_back({m, k});
    }
  for (auto& kv : faces) {
    if (kv.second.size() > 2) {
      *err = "a face is shared by more than two macros";
      return ELM_ERR_TOPOLOGY;
    }
    if (kv.second.size() == 2) {
      auto a = kv.second[0], b = kv.second[1];
      me->geo[a.first].nb[a.second] = int32_t(b.first);
      me->geo[b.first].nb[b.second] = int32_t(a.first);
    }
  }
  // Exact lattice frame changes across faces (FaceXform): A = J_mm^{-1} J_m
  // = NJinv_mm J_m / N and b = NJinv_mm (v0_m - v0_mm), kept only when every
  // entry is exactly an integer in FP64 and small.
  for (int64_t m = 0; m < nm; ++m) {
    MacroGeo& g = me->geo[m];
    std::memset(&g.x, 0, sizeof(g.x));
    for (int k = 0; k <= d; ++k) {
      const int64_t mm = g.nb[k];
      if (mm < 0) continue;
      const MacroGeo& h = me->geo[mm];
      bool ok = true;
      double A[9] = {0}, b[3] = {0};
      for (int r = 0; r < d; ++r) {
        for (int c = 0; c < d; ++c) {
          double s = 0.0;
          for (int j = 0; j < d; ++j) s += h.NJinv[r * 3 + j] * g.J[j * 3 + c];
          A[r * 3 + c] = s / double(me->N);
        }
        double t = 0.0;
        for (int j = 0; j < d; ++j) t += h.NJinv[r * 3 + j] * (g.v0[j] - h.v0[j]);
        b[r] = t;
      }
      for (int r = 0; r < d && ok; ++r) {
        ok = b[r] == std::nearbyint(b[r]) && std::fabs(b[r]) < double(1 << 20);
        for (int c = 0; c < d && ok; ++c)
          ok = A[r * 3 + c] == std::nearbyint(A[r * 3 + c]) && std::fabs(A[r * 3 + c]) <= 8.0;
      }
      if (!ok) continue;
      for (int r = 0; r < d; ++r) {
        for (int c = 0; c < d; ++c) g.x.A[k][r * 3 + c] = int8_t(A[r * 3 + c]);
        g.x.b[k][r] = int32_t(b[r]);
      }
      g.x.exact |= 1 << k;
    }
  }

  // Storage layout and interface owners.  Lattice point p of macro m sits at
  // slot m * npm + packed(p); its integer barycentric weights are
  // (M - p1, p1 - p2, p2 - p3, p3).  Interior points are owned by their macro;
  // interface points by the first macro that holds them.
  const int M = me->M;
  me->n_ghost = 0;
  me->unique_map.assign(me->n_storage, -1);
  me->owner.clear();
  me->owner.reserve(me->n_storage);
  std::unordered_map<NodeKey, int64_t, NodeKeyHash> shared;
  int64_t next = 0;
  for (int64_t m = 0; m < nm; ++m) {
    int64_t slot = m * me->npm;
    int p[3] = {0, 0, 0};
    auto visit = [&]() {
      int pp[5] = {M, p[0], p[1], p[2], 0};
      if (d == 2) pp[3] = 0;
      int w[4];
      bool interior = true;
      for (int k = 0; k <= d; ++k) {
        w[k] = pp[k] - pp[k + 1];
        interior = interior && w[k] > 0;
      }
      if (interior) {
        me->unique_map[slot] = next++;
        me->owner.push_back(slot);
      } else {
        NodeKey key;
        key.fill(-1);
        int n = 0;
        for (int k = 0; k <= d; ++k)
          if (w[k] > 0) {
            key[n++] = verts[m][k];
            key[n++] = w[k];
          }
        auto it = shared.find(key);
        if (it == shared.end()) {
          shared.emplace(key, next);
          me->unique_map[slot] = next++;
          me->owner.push_back(slot);
        } else {
          me->unique_map[slot] = it->second;
          ++me->n_ghost;
        }
      }
      ++slot;
    };
    if (d == 2) {
      for (p[0] = 0; p[0] <= M; ++p[0])
        for (p[1] = 0; p[1] <= p[0]; ++p[1]) visit();
    } else {
      for (p[0] = 0; p[0] <= M; ++p[0])
        for (p[1] = 0; p[1] <= p[0]; ++p[1])
          for (p[2] = 0; p[2] <= p[1]; ++p[2]) visit();
    }
  }
  me->n_unique = next;

  if (me->host_only) return ELM_OK;

  // Device tables.
  // Owner records (elm::pack_owner): the owner macro and its lattice point.
  std::vector<int64_t> slot_p(me->npm);
  {
    int64_t k = 0;
    if (d == 2) {
      for (int p1 = 0; p1 <= M; ++p1)
        for (int p2 = 0; p2 <= p1; ++p2) slot_p[k++] = elm::pack_owner(0, p1, p2, 0);
    } else {
      for (int p1 = 0; p1 <= M; ++p1)
        for (int p2 = 0; p2 <= p1; ++p2)
          for (int p3 = 0; p3 <= p2; ++p3) slot_p[k++] = elm::pack_owner(0, p1, p2, p3);
    }
  }
  std::vector<int64_t> owner_mp(me->n_unique);
  for (int64_t u = 0; u < me->n_unique; ++u) {
    const int64_t m = me->owner[u] / me->npm;
    owner_mp[u] = elm::pack_owner(m, 0, 0, 0) | slot_p[me->owner[u] - m * me->npm];
  }
  // Work list: each slab p1 of each macro split into runs of kAdvectThreads
  // nodes (slab p1 holds (p1+1)(p1+2)/2 nodes in 3D, p1+1 in 2D).
  std::vector<int4> chunks;
  for (int64_t m = 0; m < nm; ++m)
    for (int p1 = 0; p1 <= M; ++p1) {
      const int len = d == 3 ? (p1 + 1) * (p1 + 2) / 2 : p1 + 1;
      for (int i0 = 0; i0 < len; i0 += kAdvectThreads)
        chunks.push_back(make_int4(int(m), p1, i0, std::min(kAdvectThreads, len - i0)));
    }
  me->n_chunks = int64_t(chunks.size());
  me->chunks = chunks;
  // Interface copies other than the owner's, in storage order.  The owner is
  // the first macro holding the node, so its slot (and its work-list chunk)
  // always comes before the copy's.
  me->ghosts.clear();
  me->ghosts.reserve(size_t(me->n_ghost));
  for (int64_t s = 0; s < me->n_storage; ++s) {
    const int64_t o = me->owner[size_t(me->unique_map[size_t(s)])];
    if (o != s) me->ghosts.push_back(make_int2(int(s), int(o)));
  }
  auto upload = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (bytes == 0) { *dst = nullptr; return true; }
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  std::vector<MacroGeo32> g32(nm);
  auto split = [](double x, float* hi, float* lo) {
    *hi = float(x);
    *lo = float(x - double(*hi));
  };
  for (int64_t m = 0; m < nm; ++m) {
    for (int k = 0; k < 9; ++k) {
      split(me->geo[m].NJinv[k], &g32[m].NJinv[k], &g32[m].NJinv_lo[k]);
      split(me->geo[m].J[k], &g32[m].J[k], &g32[m].J_lo[k]);
    }
    for (int k = 0; k < 3; ++k) split(me->geo[m].v0[k], &g32[m].v0[k], &g32[m].v0_lo[k]);
    for (int k = 0; k < 4; ++k) g32[m].nb[k] = me->geo[m].nb[k];
    g32[m].x = me->geo[m].x;
  }
  bool ok = upload((void**)&me->d_geo, me->geo.data(), sizeof(MacroGeo) * nm) &&
            upload((void**)&me->d_geo32, g32.data(), sizeof(MacroGeo32) * nm) &&
            upload((void**)&me->d_unique_map, me->unique_map.data(), sizeof(int64_t) * me->n_storage) &&
            upload((void**)&me->d_owner, me->owner.data(), sizeof(int64_t) * me->n_unique) &&
            upload((void**)&me->d_owner_mp, owner_mp.data(), sizeof(int64_t) * me->n_unique) &&
            upload((void**)&me->d_chunks, chunks.data(), sizeof(int4) * chunks.size()) &&
            upload((void**)&me->d_ghosts, me->ghosts.data(), sizeof(int2) * me->ghosts.size()) &&
            cudaMalloc(&me->d_u4[0], size_t(me->n_storage) * 4 * (precision == ELM_FP64 ? 8 : 4)) == cudaSuccess &&
            cudaMalloc(&me->d_u4[1], size_t(me->n_storage) * 4 * (precision == ELM_FP64 ? 8 : 4)) == cudaSuccess &&
            (!me->with_adjoint ||
             (cudaMalloc((void**)&me->d_acc_T, sizeof(unsigned long long) * me->n_storage) == cudaSuccess &&
              cudaMalloc((void**)&me->d_acc_U, sizeof(unsigned long long) * me->n_storage * d * 2) == cudaSuccess &&
              cudaMalloc((void**)&me->d_adj_stat, sizeof(unsigned long long) * me->n_storage * 6) == cudaSuccess &&
              cudaMalloc((void**)&me->d_adj_kexp, sizeof(int) * me->n_storage * 3) == cudaSuccess)) &&
            cudaMalloc((void**)&me->d_status, sizeof(unsigned)) == cudaSuccess &&
            cudaMemset(me->d_status, 0, sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    *err = std::string("device table upload failed: ") + cudaGetErrorString(cudaGetLastError());
    return ELM_ERR_CUDA;
  }
  if (me->with_diffusion) return build_diffusion(me, err);
  return ELM_OK;
}

}  // namespace elm
