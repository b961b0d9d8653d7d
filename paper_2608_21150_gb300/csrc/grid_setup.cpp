// Host-side grid validation and geometric factors (row A0: setup, not timed).
//
// The paper gives the grid (icosahedral RnBm, Sec. 5.1) and the C-ABI
// problem of passing connectivity and geometry once at setup (Sec. 4.3.1),
// but no discretisation formula.  The factors built here follow the
// ICON-type reading documented in the design notes of this repository:
// spherical-triangle cell areas, great-circle primal and dual edge lengths,
// dual areas as fans of (vertex, circumcentre, circumcentre) triangles,
// normals from cell c0 to c1, tangent t = r x n, Perot reconstructions for
// the tangential wind and the vertex velocity, Green-Gauss cell gradients,
// and area-weighted edge->cell and cell->vertex interpolation.
#include <cmath>
#include <cstdio>
#include <string>

#include "internal.h"

namespace icon {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return (1.0 / norm(a)) * a; }
inline V3 tangential(V3 v, V3 x) { return v - dot(v, x) * x; }
inline double arc(V3 p, V3 q) { return std::atan2(norm(cross(p, q)), dot(p, q)); }
inline double tri_area(V3 p, V3 q, V3 r) {
  double num = std::fabs(dot(p, cross(q, r)));
  double den = 1.0 + dot(p, q) + dot(q, r) + dot(r, p);
  return 2.0 * std::atan2(num, den);
}
inline V3 at(const std::vector<double>& xyz, int i) {
  return {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
}

std::string fmt(const char* f, long a, long b = 0, long c = 0) {
  char buf[256];
  std::snprintf(buf, sizeof buf, f, a, b, c);
  return buf;
}

}  // namespace

std::string build_host_grid(const icon_grid_desc_t* d, HostGrid* g) {
  const int nc = d->n_cells, ne = d->n_edges, nv = d->n_verts, base = d->index_base;
  g->nc = nc;
  g->ne = ne;
  g->nv = nv;
  g->radius = d->sphere_radius;
  const double a = d->sphere_radius;

  auto load = [&](const int32_t* src, int n, int w, std::vector<int>& dst, int lo_ok) -> std::string {
    dst.resize((size_t)n * w);
    int hi = (&dst == &g->c2v || &dst == &g->e2v || &dst == &g->v2e ? 0 : 0);
    (void)hi;
    for (size_t i = 0; i < dst.size(); ++i) dst[i] = src[i] - base;
    (void)lo_ok;
    return "";
  };
  load(d->c2v, nc, 3, g->c2v, 0);
  load(d->c2e, nc, 3, g->c2e, 0);
  load(d->e2c, ne, 2, g->e2c, 0);
  load(d->e2v, ne, 2, g->e2v, 0);
  load(d->v2e, nv, 6, g->v2e, 1);
  load(d->v2c, nv, 6, g->v2c, 1);
  g->cell_xyz.assign(d->cell_xyz, d->cell_xyz + 3 * (size_t)nc);
  g->vert_xyz.assign(d->vert_xyz, d->vert_xyz + 3 * (size_t)nv);
  g->edge_xyz.assign(d->edge_xyz, d->edge_xyz + 3 * (size_t)ne);

  // ---------------- validation ----------------
  if (nv - ne + nc != 2) return fmt("grid is not a closed sphere: V - E + F = %ld", nv - ne + nc);
  if (3L * nc != 2L * ne) return fmt("grid is not triangular: 3*n_cells=%ld != 2*n_edges=%ld", 3L * nc, 2L * ne);
  auto in = [](int i, int n) { return i >= 0 && i < n; };
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < 3; ++j) {
      if (!in(g->c2v[3 * c + j], nv)) return fmt("c2v[%ld][%ld] out of range", c, j);
      if (!in(g->c2e[3 * c + j], ne)) return fmt("c2e[%ld][%ld] out of range", c, j);
    }
  for (int e = 0; e < ne; ++e) {
    for (int j = 0; j < 2; ++j) {
      if (!in(g->e2c[2 * e + j], nc)) return fmt("e2c[%ld][%ld] out of range", e, j);
      if (!in(g->e2v[2 * e + j], nv)) return fmt("e2v[%ld][%ld] out of range", e, j);
    }
    if (g->e2c[2 * e] == g->e2c[2 * e + 1]) return fmt("edge %ld has the same cell twice", e);
    if (g->e2v[2 * e] == g->e2v[2 * e + 1]) return fmt("edge %ld has the same vertex twice", e);
    for (int j = 0; j < 2; ++j) {
      int c = g->e2c[2 * e + j];
      for (int i = 0; i < 2; ++i) {
        int v = g->e2v[2 * e + i];
        if (g->c2v[3 * c] != v && g->c2v[3 * c + 1] != v && g->c2v[3 * c + 2] != v)
          return fmt("vertex %ld of edge %ld is not a vertex of its cell %ld", v, e, c);
      }
    }
  }
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < 3; ++j) {
      int e = g->c2e[3 * c + j];
      if (g->e2c[2 * e] != c && g->e2c[2 * e + 1] != c)
        return fmt("cell %ld lists edge %ld which does not list it back", c, e);
    }
  // vertex degrees from the edges' own vertex lists: every vertex row must
  // hold each of its edges exactly once (a repeated entry would drop another
  // edge from the vertex's circulation and average)
  std::vector<int> degree(nv, 0);
  for (int e = 0; e < ne; ++e) {
    ++degree[g->e2v[2 * e]];
    ++degree[g->e2v[2 * e + 1]];
  }
  for (int v = 0; v < nv; ++v) {
    int ne_v = 0, nc_v = 0;
    for (int j = 0; j < 6; ++j) {
      int e = g->v2e[6 * v + j], c = g->v2c[6 * v + j];
      if (e != -1) {
        if (!in(e, ne)) return fmt("v2e[%ld][%ld] out of range", v, j);
        if (g->e2v[2 * e] != v && g->e2v[2 * e + 1] != v)
          return fmt("vertex %ld lists edge %ld which does not list it back", v, e);
        for (int i = 0; i < j; ++i)
          if (g->v2e[6 * v + i] == e) return fmt("vertex %ld lists edge %ld twice", v, e);
        ++ne_v;
      }
      if (c != -1) {
        if (!in(c, nc)) return fmt("v2c[%ld][%ld] out of range", v, j);
        if (g->c2v[3 * c] != v && g->c2v[3 * c + 1] != v && g->c2v[3 * c + 2] != v)
          return fmt("vertex %ld lists cell %ld which does not list it back", v, c);
        for (int i = 0; i < j; ++i)
          if (g->v2c[6 * v + i] == c) return fmt("vertex %ld lists cell %ld twice", v, c);
        ++nc_v;
      }
    }
    if (ne_v < 3 || nc_v != ne_v) return fmt("vertex %ld has %ld edges and %ld cells", v, ne_v, nc_v);
    if (ne_v != degree[v]) return fmt("vertex %ld lists %ld edges but %ld edges end at it", v, ne_v, degree[v]);
  }
  auto unit_ok = [](const std::vector<double>& xyz) {
    for (size_t i = 0; i < xyz.size() / 3; ++i) {
      double n2 = xyz[3 * i] * xyz[3 * i] + xyz[3 * i + 1] * xyz[3 * i + 1] + xyz[3 * i + 2] * xyz[3 * i + 2];
      if (!(std::fabs(n2 - 1.0) < 1e-6)) return false;
    }
    return true;
  };
  if (!unit_ok(g->cell_xyz) || !unit_ok(g->vert_xyz) || !unit_ok(g->edge_xyz))
    return "coordinates must be finite unit vectors";
  if (!(a > 0.0) || !std::isfinite(a)) return "sphere_radius must be positive";

  // ---------------- derived connectivity ----------------
  g->c2e2c.resize(3 * (size_t)nc);
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < 3; ++j) {
      int e = g->c2e[3 * c + j];
      g->c2e2c[3 * c + j] = g->e2c[2 * e] == c ? g->e2c[2 * e + 1] : g->e2c[2 * e];
    }
  std::vector<V3> nrm(ne), tng(ne);
  g->e2v_t.resize(2 * (size_t)ne);
  g->e2c2v.resize(4 * (size_t)ne);
  g->e2c2e.resize(4 * (size_t)ne);
  for (int e = 0; e < ne; ++e) {
    V3 E = at(g->edge_xyz, e);
    int c0 = g->e2c[2 * e], c1 = g->e2c[2 * e + 1];
    nrm[e] = unit(tangential(at(g->cell_xyz, c1) - at(g->cell_xyz, c0), E));
    tng[e] = cross(E, nrm[e]);
    int va = g->e2v[2 * e], vb = g->e2v[2 * e + 1];
    if (dot(at(g->vert_xyz, vb) - at(g->vert_xyz, va), tng[e]) < 0) std::swap(va, vb);
    g->e2v_t[2 * e] = va;
    g->e2v_t[2 * e + 1] = vb;
    g->e2c2v[4 * e] = va;
    g->e2c2v[4 * e + 1] = vb;
    for (int s = 0; s < 2; ++s) {
      int c = g->e2c[2 * e + s];
      int opp = -1, k = 0;
      for (int j = 0; j < 3; ++j) {
        int v = g->c2v[3 * c + j];
        if (v != va && v != vb) opp = v;
        int ej = g->c2e[3 * c + j];
        if (ej != e && k < 2) g->e2c2e[4 * e + 2 * s + k++] = ej;
      }
      if (opp < 0 || k != 2) return fmt("cell %ld of edge %ld is degenerate", c, e);
      g->e2c2v[4 * e + 2 + s] = opp;
    }
  }

  // ---------------- metric factors ----------------
  g->cell_area.resize(nc);
  g->edge_length.resize(ne);
  g->dual_length.resize(ne);
  g->dual_area.assign(nv, 0.0);
  g->edge_area.resize(ne);
  double area_sum = 0.0;
  for (int c = 0; c < nc; ++c) {
    g->cell_area[c] = a * a * tri_area(at(g->vert_xyz, g->c2v[3 * c]), at(g->vert_xyz, g->c2v[3 * c + 1]),
                                       at(g->vert_xyz, g->c2v[3 * c + 2]));
    area_sum += g->cell_area[c];
  }
  g->mean_area = area_sum / nc;
  for (int e = 0; e < ne; ++e) {
    g->edge_length[e] = a * arc(at(g->vert_xyz, g->e2v[2 * e]), at(g->vert_xyz, g->e2v[2 * e + 1]));
    g->dual_length[e] = a * arc(at(g->cell_xyz, g->e2c[2 * e]), at(g->cell_xyz, g->e2c[2 * e + 1]));
    g->edge_area[e] = g->edge_length[e] * g->dual_length[e];
  }
  for (int v = 0; v < nv; ++v) {
    V3 P = at(g->vert_xyz, v);
    double s = 0.0;
    for (int j = 0; j < 6; ++j) {
      int e = g->v2e[6 * v + j];
      if (e < 0) continue;
      s += tri_area(P, at(g->cell_xyz, g->e2c[2 * e]), at(g->cell_xyz, g->e2c[2 * e + 1]));
    }
    g->dual_area[v] = a * a * s;
  }

  // cell coefficients and frames
  g->div_c.resize(3 * (size_t)nc);
  g->lap_c.resize(3 * (size_t)nc);
  g->e2c_w.resize(3 * (size_t)nc);
  g->grad_c.resize(6 * (size_t)nc);
  std::vector<V3> f1(nc), f2(nc);
  for (int c = 0; c < nc; ++c) {
    V3 C = at(g->cell_xyz, c);
    f1[c] = unit(tangential(at(g->edge_xyz, g->c2e[3 * c]) - C, C));
    f2[c] = cross(C, f1[c]);
    double A = g->cell_area[c], qs = 0.0, q[3];
    for (int j = 0; j < 3; ++j) {
      int e = g->c2e[3 * c + j];
      double sgn = g->e2c[2 * e] == c ? 1.0 : -1.0;
      double l = g->edge_length[e], dd = g->dual_length[e];
      g->div_c[3 * c + j] = sgn * l / A;
      g->lap_c[3 * c + j] = l / (dd * A);
      q[j] = l * (a * arc(C, at(g->edge_xyz, e))) / (2.0 * A);
      qs += q[j];
      // edge value = linear interpolation along the dual edge to the edge midpoint
      int cn = g->c2e2c[3 * c + j];
      double r_self = arc(C, at(g->edge_xyz, e)), r_nbr = arc(at(g->cell_xyz, cn), at(g->edge_xyz, e));
      double w_self = r_nbr / (r_self + r_nbr);
      V3 w = (sgn * l / A) * nrm[e];
      double wx = dot(w, f1[c]), wy = dot(w, f2[c]);
      // gradient = sum_j G_j (psi_nbr_j - psi_c): exact for constants on the sphere
      g->grad_c[6 * c + 2 * j] = (1.0 - w_self) * wx;
      g->grad_c[6 * c + 2 * j + 1] = (1.0 - w_self) * wy;
    }
    for (int j = 0; j < 3; ++j) g->e2c_w[3 * c + j] = q[j] / qs;
  }

  // cell velocity (Perot reconstruction) as east/north components: u = sum_j ce_j vn_j,
  // v = sum_j cn_j vn_j (corrector features)
  g->uv_c.resize(6 * (size_t)nc);
  for (int c = 0; c < nc; ++c) {
    V3 C = at(g->cell_xyz, c);
    V3 east = unit(cross(V3{0.0, 0.0, 1.0}, C));
    V3 north = cross(C, east);
    for (int j = 0; j < 3; ++j) {
      int e = g->c2e[3 * c + j];
      double sgn = g->e2c[2 * e] == c ? 1.0 : -1.0;
      V3 dx = tangential(a * (at(g->edge_xyz, e) - C), C);
      double coef = sgn * g->edge_length[e] / g->cell_area[c];
      g->uv_c[6 * c + 2 * j] = coef * dot(dx, east);
      g->uv_c[6 * c + 2 * j + 1] = coef * dot(dx, north);
    }
  }

  // edge coefficients
  g->inv_d.resize(ne);
  g->inv_l.resize(ne);
  g->vt_w.resize(5 * (size_t)ne);
  g->upw.resize(12 * (size_t)ne);
  g->nt.resize(6 * (size_t)ne);
  g->inv_dn.resize(ne);
  g->coriolis_z.resize(ne);
  for (int e = 0; e < ne; ++e) {
    V3 E = at(g->edge_xyz, e);
    g->inv_d[e] = 1.0 / g->dual_length[e];
    g->inv_l[e] = 1.0 / g->edge_length[e];
    g->coriolis_z[e] = E.z;
    double* w = &g->vt_w[5 * (size_t)e];
    for (int j = 0; j < 5; ++j) w[j] = 0.0;
    for (int s = 0; s < 2; ++s) {
      int c = g->e2c[2 * e + s];
      V3 C = at(g->cell_xyz, c);
      double A = g->cell_area[c];
      int k = 0;
      for (int j = 0; j < 3; ++j) {
        int ej = g->c2e[3 * c + j];
        double sgn = g->e2c[2 * ej] == c ? 1.0 : -1.0;
        V3 dx = tangential(a * (at(g->edge_xyz, ej) - C), C);
        double coef = 0.5 * sgn * g->edge_length[ej] / A * dot(tng[e], dx);
        if (ej == e)
          w[0] += coef;
        else
          w[1 + 2 * s + k++] += coef;
      }
      V3 dx = a * (E - C);
      double* u = &g->upw[12 * (size_t)e + 6 * s];
      u[0] = dot(dx, f1[c]);
      u[1] = dot(dx, f2[c]);
      u[2] = dot(nrm[e], f1[c]);
      u[3] = dot(nrm[e], f2[c]);
      u[4] = dot(tng[e], f1[c]);
      u[5] = dot(tng[e], f2[c]);
    }
    double* nt = &g->nt[6 * (size_t)e];
    nt[0] = nrm[e].x; nt[1] = nrm[e].y; nt[2] = nrm[e].z;
    nt[3] = tng[e].x; nt[4] = tng[e].y; nt[5] = tng[e].z;
    g->inv_dn[e] = 1.0 / (a * arc(at(g->vert_xyz, g->e2c2v[4 * e + 2]), at(g->vert_xyz, g->e2c2v[4 * e + 3])));
  }

  // vertex coefficients
  g->curl_v.assign(6 * (size_t)nv, 0.0);
  g->c2v_w.assign(6 * (size_t)nv, 0.0);
  g->uv_w.assign(18 * (size_t)nv, 0.0);
  for (int v = 0; v < nv; ++v) {
    V3 P = at(g->vert_xyz, v);
    double rs = 0.0;
    for (int j = 0; j < 6; ++j) {
      int e = g->v2e[6 * v + j];
      if (e >= 0) {
        double sgn = dot(P - at(g->edge_xyz, e), tng[e]) > 0 ? 1.0 : -1.0;
        double coef = sgn * g->dual_length[e] / g->dual_area[v];
        g->curl_v[6 * v + j] = coef;
        V3 M = unit(at(g->cell_xyz, g->e2c[2 * e]) + at(g->cell_xyz, g->e2c[2 * e + 1]));
        V3 U = cross(P, tangential(coef * (a * (M - P)), P));
        g->uv_w[18 * v + 3 * j] = U.x;
        g->uv_w[18 * v + 3 * j + 1] = U.y;
        g->uv_w[18 * v + 3 * j + 2] = U.z;
      }
      int c = g->v2c[6 * v + j];
      if (c >= 0) {
        V3 C = at(g->cell_xyz, c);
        V3 m[2];
        int k = 0;
        for (int i = 0; i < 3; ++i) {
          int o = g->c2v[3 * c + i];
          if (o != v && k < 2) m[k++] = unit(at(g->vert_xyz, o) + P);
        }
        double kite = tri_area(P, m[0], C) + tri_area(P, C, m[1]);
        g->c2v_w[6 * v + j] = kite;
        rs += kite;
      }
    }
    for (int j = 0; j < 6; ++j) g->c2v_w[6 * v + j] /= rs;
    // pads point at a valid index (weight 0)
    for (int j = 0; j < 6; ++j) {
      if (g->v2e[6 * v + j] < 0) g->v2e[6 * v + j] = g->v2e[6 * v];
      if (g->v2c[6 * v + j] < 0) g->v2c[6 * v + j] = g->v2c[6 * v];
    }
  }
  return "";
}

}  // namespace icon
