// Host-side tables of the fused velocity-advection kernel (rows A1-A4 in
// one launch, mixed precision over flat ground): the cells are cut into
// patches of consecutive indices (the refinement order of the grid makes
// them compact); for every patch the lists of the cells, edges and
// vertices whose values its own cells' tendencies need, with their
// connectivity in local (patch) indices, packed as 16-bit entries.
//
//   C3  the patch's own cells first, then the other cells of its edges
//   C0  C3, then the other cells around the V3 vertices (w is staged on C0)
//   E1  the edges of the C3 cells (2K and vt are formed on them)
//   V3  the vertices of the own cells' edges (vorticity, w at vertices)
//   E4  the own cells' edges (vn at half levels, the vn tendency, w's
//       horizontal advection); an edge is written by the patch of its
//       first cell only, and those edges come first
//   E0  every edge whose vn is read: E1, their four neighbours of the
//       tangential-wind stencil, and the edges around the V3 vertices
#include <algorithm>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace icon {

std::string build_va_patches(const HostGrid& g, int P, HostVaPatches* out) {
  if (P < 1) return "patch size must be positive";
  HostVaPatches& t = *out;
  t = HostVaPatches{};
  t.P = P;
  const int nc = g.nc;
  const int np = (nc + P - 1) / P;
  t.n_patches = np;
  for (auto* o : {&t.off_e0, &t.off_e1, &t.off_c0, &t.off_v3, &t.off_e4}) o->assign(1, 0);
  t.own_i.assign(4 * (size_t)nc, 0);
  std::unordered_map<int, int> le0, le1, lc0, lv3, le4;
  auto add = [](std::unordered_map<int, int>& m, std::vector<int>& v, int x) {
    auto it = m.find(x);
    if (it != m.end()) return it->second;
    const int i = (int)v.size();
    m.emplace(x, i);
    v.push_back(x);
    return i;
  };
  auto u16 = [](int x) { return (uint16_t)x; };
  for (int p = 0; p < np; ++p) {
    const int c_begin = p * P, c_end = std::min(nc, c_begin + P);
    le0.clear();
    le1.clear();
    lc0.clear();
    lv3.clear();
    le4.clear();
    std::vector<int> c0, e1, v3, e4, e0;
    for (int c = c_begin; c < c_end; ++c) add(lc0, c0, c);
    for (int c = c_begin; c < c_end; ++c)
      for (int j = 0; j < 3; ++j) add(le4, e4, g.c2e[3 * (size_t)c + j]);
    // the edges this patch writes (first cell in the patch) first
    std::stable_partition(e4.begin(), e4.end(), [&](int e) { return g.e2c[2 * (size_t)e] / P == p; });
    int nw4 = 0;
    le4.clear();
    for (int i = 0; i < (int)e4.size(); ++i) {
      le4.emplace(e4[i], i);
      if (g.e2c[2 * (size_t)e4[i]] / P == p) nw4 = i + 1;
    }
    t.n_w4.push_back(nw4);
    for (int e : e4) {
      add(lc0, c0, g.e2c[2 * (size_t)e]);
      add(lc0, c0, g.e2c[2 * (size_t)e + 1]);
      add(lv3, v3, g.e2v[2 * (size_t)e]);
      add(lv3, v3, g.e2v[2 * (size_t)e + 1]);
    }
    const int nc3 = (int)c0.size();
    for (int i = 0; i < nc3; ++i)
      for (int j = 0; j < 3; ++j) add(le1, e1, g.c2e[3 * (size_t)c0[i] + j]);
    for (int e : e1) {
      add(le0, e0, e);
      for (int j = 0; j < 4; ++j) add(le0, e0, g.e2c2e[4 * (size_t)e + j]);
    }
    for (int v : v3)
      for (int j = 0; j < 6; ++j) {
        add(le0, e0, g.v2e[6 * (size_t)v + j]);
        add(lc0, c0, g.v2c[6 * (size_t)v + j]);
      }
    if (std::max({e0.size(), c0.size(), e1.size(), v3.size(), e4.size()}) > 65535)
      return "patch lists exceed 16-bit local indices";
    t.n_c3.push_back(nc3);
    for (int e : e0) t.e0_g.push_back(e);
    for (int c : c0) t.c0_g.push_back(c);
    for (int i = 0; i < (int)c0.size(); ++i)
      for (int j = 0; j < 4; ++j) t.c3_i.push_back(i < nc3 && j < 3 ? u16(le1.at(g.c2e[3 * (size_t)c0[i] + j])) : 0);
    for (int e : e1) {
      t.e1_g.push_back(e);
      t.e1_i.push_back(u16(le0.at(e)));
      for (int j = 0; j < 4; ++j) t.e1_i.push_back(u16(le0.at(g.e2c2e[4 * (size_t)e + j])));
      for (int j = 5; j < 8; ++j) t.e1_i.push_back(0);
    }
    for (int v : v3) {
      t.v3_g.push_back(v);
      for (int j = 0; j < 6; ++j) t.v3_i.push_back(u16(le0.at(g.v2e[6 * (size_t)v + j])));
      for (int j = 0; j < 6; ++j) t.v3_i.push_back(u16(lc0.at(g.v2c[6 * (size_t)v + j])));
      for (int j = 12; j < 16; ++j) t.v3_i.push_back(0);
    }
    for (int e : e4) {
      t.e4_g.push_back(e);
      const int ca = g.e2c[2 * (size_t)e], cb = g.e2c[2 * (size_t)e + 1];
      t.e4_i.push_back(u16(le1.at(e)));
      t.e4_i.push_back(u16(le0.at(e)));
      t.e4_i.push_back(u16(lc0.at(ca)));
      t.e4_i.push_back(u16(lc0.at(cb)));
      t.e4_i.push_back(u16(lv3.at(g.e2v[2 * (size_t)e])));
      t.e4_i.push_back(u16(lv3.at(g.e2v[2 * (size_t)e + 1])));
      t.e4_i.push_back(0);
      t.e4_i.push_back(0);
    }
    for (int c = c_begin; c < c_end; ++c)
      for (int j = 0; j < 3; ++j) t.own_i[4 * (size_t)c + j] = u16(le4.at(g.c2e[3 * (size_t)c + j]));
    t.off_e0.push_back((int)t.e0_g.size());
    t.off_e1.push_back((int)t.e1_g.size());
    t.off_c0.push_back((int)t.c0_g.size());
    t.off_v3.push_back((int)t.v3_g.size());
    t.off_e4.push_back((int)t.e4_g.size());
    t.max_e0 = std::max(t.max_e0, (int)e0.size());
    t.max_e1 = std::max(t.max_e1, (int)e1.size());
    t.max_c3 = std::max(t.max_c3, nc3);
    t.max_c0 = std::max(t.max_c0, (int)c0.size());
    t.max_v3 = std::max(t.max_v3, (int)v3.size());
    t.max_e4 = std::max(t.max_e4, (int)e4.size());
  }
  return "";
}

}  // namespace icon
