// host_mesh_tables.h -- the tables the library uploads at mesh creation (owner
// records, the work list, the FP32 split of the macro tables, the interface
// copies, the annulus sector table), built from a host-only mesh in the same
// way, for the host builds of
// the kernels' device code (tests/kernel_host_check.cpp,
// tests/adjoint_host_check.cpp).  Test infrastructure only.
#pragma once

#include <cmath>
#include <vector>

#include "elm_internal.h"

namespace elm_host_check {

using namespace elm;

struct HostTables {
  std::vector<int64_t> owner_mp;
  std::vector<int4> chunks;
  std::vector<MacroGeo32> geo32;
  std::vector<int2> ghosts;
};

inline HostTables host_tables(const elm_mesh_s* me) {
  HostTables h;
  const int d = me->dim, M = me->M;
  std::vector<int64_t> slot_p(size_t(me->npm));
  int64_t k = 0;
  if (d == 2) {
    for (int p1 = 0; p1 <= M; ++p1)
      for (int p2 = 0; p2 <= p1; ++p2) slot_p[size_t(k++)] = pack_owner(0, p1, p2, 0);
  } else {
    for (int p1 = 0; p1 <= M; ++p1)
      for (int p2 = 0; p2 <= p1; ++p2)
        for (int p3 = 0; p3 <= p2; ++p3) slot_p[size_t(k++)] = pack_owner(0, p1, p2, p3);
  }
  h.owner_mp.resize(size_t(me->n_unique));
  for (int64_t u = 0; u < me->n_unique; ++u) {
    const int64_t m = me->owner[size_t(u)] / me->npm;
    h.owner_mp[size_t(u)] = pack_owner(m, 0, 0, 0) | slot_p[size_t(me->owner[size_t(u)] - m * me->npm)];
  }
  for (int64_t m = 0; m < me->n_macros; ++m)
    for (int p1 = 0; p1 <= M; ++p1) {
      const int len = d == 3 ? (p1 + 1) * (p1 + 2) / 2 : p1 + 1;
      for (int i0 = 0; i0 < len; i0 += kAdvectThreads)
        h.chunks.push_back(make_int4(int(m), p1, i0, len - i0 < kAdvectThreads ? len - i0 : kAdvectThreads));
    }
  for (int64_t s = 0; s < me->n_storage; ++s) {
    const int64_t o = me->owner[size_t(me->unique_map[size_t(s)])];
    if (o != s) h.ghosts.push_back(make_int2(int(s), int(o)));
  }
  h.geo32.resize(size_t(me->n_macros));
  auto split = [](double x, float* hi, float* lo) {
    *hi = float(x);
    *lo = float(x - double(*hi));
  };
  for (int64_t m = 0; m < me->n_macros; ++m) {
    const MacroGeo& g = me->geo[size_t(m)];
    MacroGeo32& g32 = h.geo32[size_t(m)];
    for (int q = 0; q < 9; ++q) {
      split(g.NJinv[q], &g32.NJinv[q], &g32.NJinv_lo[q]);
      split(g.J[q], &g32.J[q], &g32.J_lo[q]);
    }
    for (int q = 0; q < 3; ++q) split(g.v0[q], &g32.v0[q], &g32.v0_lo[q]);
    for (int q = 0; q < 4; ++q) g32.nb[q] = g.nb[q];
    g32.x = g.x;
  }
  return h;
}

// Unit vectors at the sector boundaries theta0 + k 2 pi / n, k = 0..n ([n + 1][2];
// the last repeats the first), the annulus blending's sector table.
inline std::vector<double> sector_table(int n, double theta0) {
  std::vector<double> sec(size_t(2 * (n + 1)));
  const double delta = 2.0 * 3.14159265358979323846 / n;
  for (int k = 0; k <= n; ++k) {
    sec[size_t(2 * k)] = std::cos(theta0 + (k % n) * delta);
    sec[size_t(2 * k + 1)] = std::sin(theta0 + (k % n) * delta);
  }
  return sec;
}

}  // namespace elm_host_check
