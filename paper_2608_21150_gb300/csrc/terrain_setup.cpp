// Host set-up of the vertical coordinate (row A0): per-column metrics and
// reference state, and the terrain-following coordinate's edge metrics and
// slopes (readings of an ICON-type scheme; the paper's dycore runs over real
// topography, Sec. 4.1, but states no formula).
//   * per column: full level = mid-point, dz, interior half-level spacing and
//     interpolation weight, reference state theta_ref = T0 exp(z/H) with
//     exner_ref integrated upward in exact discrete balance, Rayleigh factors,
//     and the column solve's coefficients;
//   * at edges: heights are the mean of the two cells' (layer thickness and
//     interpolation weights from them); normal slopes (z_c1 - z_c0)/d_e on
//     half and full levels; tangential slopes along t_e from vertex heights,
//     each one adjacent cell's height plus the kite-weighted offsets of all
//     of them (exactly flat where the cells' heights agree);
//   * the true-horizontal pressure gradient's vertical spacing per cell:
//     centred, one-sided at the top and the ground;
//   * the ratio of each edge's layer thickness to its cell's, carried by the
//     horizontal fluxes.
#include <cmath>
#include <string>
#include <algorithm>
#include <vector>

#include "internal.h"

namespace icon {

void column_metrics(const double* z, int nlev, const icon_dycore_params_t& p, const Scalars& s, ColumnMetrics* m) {
  m->z_mc.assign(nlev, 0.0);
  m->dz.assign(nlev, 0.0);
  m->inv_dz.assign(nlev, 0.0);
  m->inv_dzh.assign(nlev + 1, 0.0);
  m->wgt.assign(nlev + 1, 0.0);
  m->dref.assign(nlev + 1, 0.0);
  m->ray.assign(nlev + 1, 1.0);
  m->theta_ref.assign(nlev, 0.0);
  m->exner_ref.assign(nlev, 0.0);
  m->colc.assign(8 * (size_t)(nlev + 1), 0.0);
  std::vector<double>& z_mc = m->z_mc;
  for (int k = 0; k < nlev; ++k) {
    z_mc[k] = 0.5 * (z[k] + z[k + 1]);
    m->dz[k] = z[k] - z[k + 1];
    m->inv_dz[k] = 1.0 / m->dz[k];
  }
  for (int k = 1; k < nlev; ++k) {
    m->inv_dzh[k] = 1.0 / (z_mc[k - 1] - z_mc[k]);
    m->wgt[k] = (z[k] - z_mc[k]) / (z_mc[k - 1] - z_mc[k]);
  }
  const double T0 = p.ref_T0, H = p.cpd * T0 / p.grav;
  for (int k = 0; k < nlev; ++k) m->theta_ref[k] = T0 * std::exp(z_mc[k] / H);
  m->exner_ref[nlev - 1] = std::exp(-z_mc[nlev - 1] / H);
  for (int k = nlev - 1; k >= 1; --k) {
    double th_ic = m->wgt[k] * m->theta_ref[k - 1] + (1.0 - m->wgt[k]) * m->theta_ref[k];
    m->exner_ref[k - 1] = m->exner_ref[k] - p.grav * (z_mc[k - 1] - z_mc[k]) / (p.cpd * th_ic);
  }
  for (int k = 1; k < nlev; ++k) m->dref[k] = (m->exner_ref[k - 1] - m->exner_ref[k]) * m->inv_dzh[k];
  if (p.rayleigh_coeff > 0.0) {
    const double top = z[0], zd = p.damp_height;
    for (int k = 0; k <= nlev; ++k)
      if (z[k] > zd) {
        double sn = std::sin(0.5 * M_PI * (z[k] - zd) / (top - zd));
        m->ray[k] = 1.0 / (1.0 + s.dt_s * p.rayleigh_coeff * sn * sn);
      }
  }
  const double dts = s.dt_s, beta = s.beta;
  for (int k = 0; k <= nlev; ++k) {
    double* c = &m->colc[8 * (size_t)k];
    if (k < nlev) {
      c[0] = dts * s.rd_o_cvd / m->dz[k];
      c[1] = dts * (1.0 - beta) / m->dz[k];
      c[2] = dts * beta / m->dz[k];
    }
    if (k >= 1 && k < nlev) {
      c[4] = dts * p.cpd * m->dref[k];
      c[5] = dts * p.cpd * beta * m->inv_dzh[k];
      c[6] = m->wgt[k];
      c[7] = 1.0 - m->wgt[k];
      c[3] = c[6] * m->theta_ref[k - 1] + c[7] * m->theta_ref[k];
    }
  }
}

std::string build_terrain(const HostGrid& g, int nlev, const double* z_ifc, const icon_dycore_params_t& p,
                          const Scalars& s, HostTerrain* t) {
  const int nc = g.nc, ne = g.ne, nv = g.nv, nlevp = nlev + 1;
  const size_t cf = (size_t)nc * nlev, ch = (size_t)nc * nlevp;
  for (int c = 0; c < nc; ++c) {
    const double* z = z_ifc + (size_t)c * nlevp;
    for (int k = 0; k <= nlev; ++k)
      if (!std::isfinite(z[k])) return "z_ifc not finite in column " + std::to_string(c);
    for (int k = 0; k < nlev; ++k)
      if (!(z[k] > z[k + 1])) return "z_ifc must decrease in every column (column " + std::to_string(c) + ")";
    if (z[0] != z_ifc[0]) return "the model top z_ifc[c][0] must be the same in every column";
  }
  t->exner_ref_c.assign(cf, 0.0);
  t->theta_ref_c.assign(cf, 0.0);
  t->dz_c.assign(cf, 0.0);
  t->inv_dzm_c.assign(cf, 0.0);
  t->inv_dzh_c.assign(ch, 0.0);
  t->colt.assign(12 * ch, 0.0);
  std::vector<double> z_mc(cf);
  ColumnMetrics m;
  for (int c = 0; c < nc; ++c) {
    column_metrics(z_ifc + (size_t)c * nlevp, nlev, p, s, &m);
    for (int k = 0; k < nlev; ++k) {
      const size_t i = (size_t)c * nlev + k;
      z_mc[i] = m.z_mc[k];
      t->exner_ref_c[i] = m.exner_ref[k];
      t->theta_ref_c[i] = m.theta_ref[k];
      t->dz_c[i] = m.dz[k];
      const int km = k > 0 ? k - 1 : 0, kp = k + 1 < nlev ? k + 1 : nlev - 1;
      t->inv_dzm_c[i] = 1.0 / (m.z_mc[km] - m.z_mc[kp]);
    }
    for (int k = 0; k <= nlev; ++k) {
      t->inv_dzh_c[(size_t)c * nlevp + k] = m.inv_dzh[k];
      auto slot = [&](int j) -> double& { return t->colt[((size_t)j * nlevp + k) * nc + c]; };
      for (int j = 0; j < 8; ++j) slot(j) = m.colc[8 * (size_t)k + j];
      if (k < nlev) {
        slot(8) = m.exner_ref[k];
        slot(9) = m.theta_ref[k];
        slot(10) = m.dz[k];
      }
      slot(11) = m.ray[k];
      if (m.ray[k] != 1.0) t->n_ray = std::max(t->n_ray, k + 1);
    }
  }
  // edges: heights the mean of the two cells'
  t->wgt_e.assign((size_t)ne * nlevp, 0.0);
  t->ddxn_ifc.assign((size_t)ne * nlevp, 0.0);
  t->ddxt_ifc.assign((size_t)ne * nlevp, 0.0);
  t->inv_dz_e.assign((size_t)ne * nlev, 0.0);
  t->ddxn_mc.assign((size_t)ne * nlev, 0.0);
  std::vector<double> dz_e((size_t)ne * nlev), ze(nlevp), ze_mc(nlev);
  for (int e = 0; e < ne; ++e) {
    const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
    const double* z0 = z_ifc + (size_t)c0 * nlevp;
    const double* z1 = z_ifc + (size_t)c1 * nlevp;
    const double d = g.dual_length[e];
    for (int k = 0; k <= nlev; ++k) {
      ze[k] = 0.5 * (z0[k] + z1[k]);
      t->ddxn_ifc[(size_t)e * nlevp + k] = (z1[k] - z0[k]) / d;
    }
    for (int k = 0; k < nlev; ++k) {
      ze_mc[k] = 0.5 * (ze[k] + ze[k + 1]);
      dz_e[(size_t)e * nlev + k] = ze[k] - ze[k + 1];
      t->inv_dz_e[(size_t)e * nlev + k] = 1.0 / dz_e[(size_t)e * nlev + k];
      t->ddxn_mc[(size_t)e * nlev + k] = (z_mc[(size_t)c1 * nlev + k] - z_mc[(size_t)c0 * nlev + k]) / d;
    }
    for (int k = 1; k < nlev; ++k)
      t->wgt_e[(size_t)e * nlevp + k] = (ze[k] - ze_mc[k]) / (ze_mc[k - 1] - ze_mc[k]);
  }
  // vertex heights: one adjacent cell's plus the weighted offsets of all
  std::vector<double> zv((size_t)nv * nlevp);
  for (int v = 0; v < nv; ++v) {
    const double* first = z_ifc + (size_t)g.v2c[6 * v] * nlevp;
    for (int k = 0; k <= nlev; ++k) {
      double x = first[k];
      for (int j = 0; j < 6; ++j) {
        const double* zc = z_ifc + (size_t)g.v2c[6 * v + j] * nlevp;
        x += g.c2v_w[6 * v + j] * (zc[k] - first[k]);
      }
      zv[(size_t)v * nlevp + k] = x;
    }
  }
  for (int e = 0; e < ne; ++e) {
    const int vm = g.e2v_t[2 * e], vp = g.e2v_t[2 * e + 1];
    const double l = g.edge_length[e];
    for (int k = 0; k <= nlev; ++k)
      t->ddxt_ifc[(size_t)e * nlevp + k] = (zv[(size_t)vp * nlevp + k] - zv[(size_t)vm * nlevp + k]) / l;
  }
  // steep terrain: edge levels whose two cells' levels are offset by more than
  // half a layer (the level of a neighbour column nearest to the edge height
  // z_e, the mean of the two cells' full-level heights, is not the same level);
  // there the pressure gradient is taken at z_e, each cell's total exner
  // interpolated by the quadratic through its three consecutive levels
  // nearest to z_e (Lagrange weights).  Heights decrease with the level, so
  // the nearest level is found by a walk that never goes back.
  // steep_idx: (edge, level, first level in e2c[0], first level in e2c[1]);
  // steep_w: the three weights in e2c[0], then the three in e2c[1]
  if (p.steep_hpg) {
    std::vector<double> ze(nlev);
    for (int e = 0; e < ne; ++e) {
      const int cs[2] = {g.e2c[2 * e], g.e2c[2 * e + 1]};
      for (int k = 0; k < nlev; ++k)
        ze[k] = 0.5 * (z_mc[(size_t)cs[0] * nlev + k] + z_mc[(size_t)cs[1] * nlev + k]);
      std::vector<int> nearest[2] = {std::vector<int>(nlev), std::vector<int>(nlev)};
      for (int sd = 0; sd < 2; ++sd) {
        const double* zc = &z_mc[(size_t)cs[sd] * nlev];
        int j = 0;
        for (int k = 0; k < nlev; ++k) {
          while (j + 1 < nlev && std::fabs(zc[j + 1] - ze[k]) < std::fabs(zc[j] - ze[k])) ++j;
          nearest[sd][k] = j;
        }
      }
      for (int k = 0; k < nlev; ++k) {
        if (nearest[0][k] == k && nearest[1][k] == k) continue;
        t->steep_idx.push_back(e);
        t->steep_idx.push_back(k);
        for (int sd = 0; sd < 2; ++sd) {
          const double* zc = &z_mc[(size_t)cs[sd] * nlev];
          int k0 = nearest[sd][k] - 1;
          k0 = k0 < 0 ? 0 : (k0 > nlev - 3 ? nlev - 3 : k0);
          t->steep_idx.push_back(k0);
          const double z[3] = {zc[k0], zc[k0 + 1], zc[k0 + 2]};
          for (int jj = 0; jj < 3; ++jj) {
            const double a = z[jj == 0 ? 1 : 0], b = z[jj == 2 ? 1 : 2];
            t->steep_w.push_back((ze[k] - a) * (ze[k] - b) / ((z[jj] - a) * (z[jj] - b)));
          }
        }
      }
    }
  }
  // flux thickness ratio of each cell's three edges
  t->fx_ratio.assign((size_t)nc * 3 * nlev, 0.0);
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < 3; ++j) {
      const int e = g.c2e[3 * c + j];
      for (int k = 0; k < nlev; ++k)
        t->fx_ratio[((size_t)c * 3 + j) * nlev + k] = dz_e[(size_t)e * nlev + k] / t->dz_c[(size_t)c * nlev + k];
    }
  return "";
}

}  // namespace icon
