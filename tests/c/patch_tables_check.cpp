// Host check of the fused velocity-advection kernel's patch tables
// (build_va_patches): every local index lies in its list and names the
// entity the global connectivity gives, the own cells come first in each
// patch's cell list, and every edge is written by exactly one patch.
// Usage: patch_tables_check GRID_FILE P; the grid file holds n_cells, n_edges,
// n_verts (int32), then c2v, c2e, e2c, e2v, v2e, v2c (int32) and the cell,
// vertex and edge positions (float64), as tests/test_patch_tables_cpu.py
// writes it.  Prints "ok" and the lists' maxima, or the first failure.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "internal.h"
using namespace icon;
template <class T> std::vector<T> rd(FILE* f, size_t n) { std::vector<T> v(n); if (fread(v.data(), sizeof(T), n, f) != n) abort(); return v; }
#define CHK(c) do { if (!(c)) { printf("FAIL %s line %d p=%d\n", #c, __LINE__, p); return 1; } } while (0)
int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int P = atoi(argv[2]);
  auto n = rd<int>(f, 3);
  int nc = n[0], ne = n[1], nv = n[2];
  auto c2v = rd<int>(f, 3 * nc), c2e = rd<int>(f, 3 * nc), e2c = rd<int>(f, 2 * ne), e2v = rd<int>(f, 2 * ne),
       v2e = rd<int>(f, 6 * nv), v2c = rd<int>(f, 6 * nv);
  auto cx = rd<double>(f, 3 * nc), vx = rd<double>(f, 3 * nv), ex = rd<double>(f, 3 * ne);
  icon_grid_desc_t d{nc, ne, nv, 0, 6.371e6, c2v.data(), c2e.data(), e2c.data(), e2v.data(), v2e.data(), v2c.data(), cx.data(), vx.data(), ex.data()};
  HostGrid g;
  std::string err = build_host_grid(&d, &g);
  if (!err.empty()) { printf("grid: %s\n", err.c_str()); return 1; }
  HostVaPatches t;
  err = build_va_patches(g, P, &t);
  if (!err.empty()) { printf("patch: %s\n", err.c_str()); return 1; }
  int p = -1;
  CHK((int)t.off_e0.size() == t.n_patches + 1 && (int)t.n_c3.size() == t.n_patches);
  CHK(t.e1_i.size() == 8 * t.e1_g.size() && t.c3_i.size() == 4 * t.c0_g.size() && t.v3_i.size() == 16 * t.v3_g.size() && t.e4_i.size() == 8 * t.e4_g.size() && t.own_i.size() == 4 * (size_t)nc);
  std::vector<int> written(ne, 0);
  for (p = 0; p < t.n_patches; ++p) {
    int e0a = t.off_e0[p], ne0 = t.off_e0[p + 1] - e0a;
    int e1a = t.off_e1[p], ne1 = t.off_e1[p + 1] - e1a;
    int c0a = t.off_c0[p], nc0 = t.off_c0[p + 1] - c0a, nc3 = t.n_c3[p];
    int v3a = t.off_v3[p], nv3 = t.off_v3[p + 1] - v3a;
    int e4a = t.off_e4[p], ne4 = t.off_e4[p + 1] - e4a;
    CHK(ne0 <= t.max_e0 && ne1 <= t.max_e1 && nc3 <= t.max_c3 && nc0 <= t.max_c0 && nv3 <= t.max_v3 && ne4 <= t.max_e4);
    CHK(nc3 <= nc0 && ne4 <= ne1);
    int cb = p * P, ncown = std::min(P, nc - cb);
    CHK(ncown <= nc3);
    for (int i = 0; i < ne0; ++i) CHK(t.e0_g[e0a + i] >= 0 && t.e0_g[e0a + i] < ne);
    for (int i = 0; i < nc0; ++i) CHK(t.c0_g[c0a + i] >= 0 && t.c0_g[c0a + i] < nc);
    for (int i = 0; i < ne1; ++i) {
      int e = t.e1_g[e1a + i];
      CHK(e >= 0 && e < ne);
      const uint16_t* x = &t.e1_i[8 * (size_t)(e1a + i)];
      for (int j = 0; j < 5; ++j) CHK(x[j] < ne0);
      CHK(t.e0_g[e0a + x[0]] == e);
      for (int j = 0; j < 4; ++j) CHK(t.e0_g[e0a + x[1 + j]] == g.e2c2e[4 * e + j]);
    }
    for (int i = 0; i < nc3; ++i) {
      int c = t.c0_g[c0a + i];
      if (i < ncown) CHK(c == cb + i);
      for (int j = 0; j < 3; ++j) { int l = t.c3_i[4 * (c0a + i) + j]; CHK(l < ne1 && t.e1_g[e1a + l] == g.c2e[3 * c + j]); }
    }
    for (int i = 0; i < nv3; ++i) {
      int v = t.v3_g[v3a + i];
      CHK(v >= 0 && v < nv);
      const uint16_t* x = &t.v3_i[16 * (size_t)(v3a + i)];
      for (int j = 0; j < 6; ++j) { CHK(x[j] < ne0 && t.e0_g[e0a + x[j]] == g.v2e[6 * v + j]); }
      for (int j = 0; j < 6; ++j) { CHK(x[6 + j] < nc0 && t.c0_g[c0a + x[6 + j]] == g.v2c[6 * v + j]); }
    }
    for (int i = 0; i < ne4; ++i) {
      int e = t.e4_g[e4a + i];
      const uint16_t* x = &t.e4_i[8 * (size_t)(e4a + i)];
      CHK(x[0] < ne1 && t.e1_g[e1a + x[0]] == e);
      CHK(x[1] < ne0 && t.e0_g[e0a + x[1]] == e);
      CHK(x[2] < nc3 && t.c0_g[c0a + x[2]] == g.e2c[2 * e]);
      CHK(x[3] < nc3 && t.c0_g[c0a + x[3]] == g.e2c[2 * e + 1]);
      CHK(x[4] < nv3 && t.v3_g[v3a + x[4]] == g.e2v[2 * e]);
      CHK(x[5] < nv3 && t.v3_g[v3a + x[5]] == g.e2v[2 * e + 1]);
      if (i < t.n_w4[p]) { written[e]++; CHK(g.e2c[2 * e] / P == p); } else CHK(g.e2c[2 * e] / P != p);
    }
    for (int c = cb; c < cb + ncown; ++c)
      for (int j = 0; j < 3; ++j) { int l = t.own_i[4 * (size_t)c + j]; CHK(l < ne4 && t.e4_g[e4a + l] == g.c2e[3 * c + j]); }
  }
  p = -1;
  for (int e = 0; e < ne; ++e) CHK(written[e] == 1);
  printf("ok %d %d %d %d %d %d %d\n", t.n_patches, t.max_e0, t.max_e1, t.max_c3, t.max_c0, t.max_v3, t.max_e4);
  return 0;
}
