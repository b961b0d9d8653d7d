// Internal data structures of the ICON-type dycore library (not part of the ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/icon_dycore.h"

namespace icon {

// Horizontal grid factors in device memory (row A0).  Index tables are
// 0-based; pad entries of the 6-wide vertex tables point at a valid index
// and carry a zero coefficient.
struct DevGrid {
  int nc, ne, nv;
  // connectivity
  const int* c2e;    // [nc*3]
  const int* c2e2c;  // [nc*3] neighbour cell across c2e[c][j]
  const int* e2c;    // [ne*2] (c0, c1): the normal points c0 -> c1
  const int* e2v;    // [ne*2] (vm, vp): the tangent points vm -> vp
  const int* e2c2v;  // [ne*4] (vm, vp, opposite vertex in c0, opposite in c1)
  const int* e2c2e;  // [ne*4] (other two edges of c0, other two of c1)
  const int* v2e;    // [nv*6]
  const int* v2c;    // [nv*6]
  // cell coefficients
  const double* div_c;   // [nc*3] s_{c,e} l_e / A_c
  const double* lap_c;   // [nc*3] l_e / (d_e A_c)
  const double* e2c_w;   // [nc*3] edge->cell interpolation weights
  const double* grad_c;  // [nc*8] Green-Gauss gradient in the cell frame: self (x,y), 3 nbrs (x,y)
  const double* k4w_c;   // [nc]   hdiff_w_k4 * A_c^2
  // edge coefficients
  const double* inv_d;   // [ne] 1/d_e
  const double* inv_l;   // [ne] 1/l_e
  const double* f_e;     // [ne] Coriolis parameter
  const double* vt_w;    // [ne*5] tangential-wind weights: self, e2c2e[0..3]
  const double* upw;     // [ne*12] per upwind side s: (dx, dy, nx, ny, tx, ty) in that cell's frame
  const double* nt;      // [ne*6] normal xyz, tangent xyz
  const double* inv_dn;  // [ne] 1/(arc between the two opposite diamond vertices)
  const double* smag_a;  // [ne] hdiff_smag_fac * A_e
  const double* k4_a;    // [ne] hdiff_k4 * A_e^2
  // vertex coefficients
  const double* curl_v;  // [nv*6] t_{v,e} d_e / A_v (0 for pads)
  const double* c2v_w;   // [nv*6] cell->vertex weights (0 for pads)
  const double* uv_w;    // [nv*6*3] vertex velocity weights (xyz per edge)
  double mean_area;
};

// Vertical metrics and reference state in device memory.
struct DevVert {
  int nlev;
  const double* dz;        // [nlev]
  const double* inv_dz;    // [nlev]
  const double* inv_dzh;   // [nlev+1] (0 at top and ground)
  const double* wgt;       // [nlev+1] weight of level k-1 at half level k (0 at ends)
  const double* theta_ref; // [nlev]
  const double* exner_ref; // [nlev]
  const double* dexner_ref_ic;  // [nlev+1]
  const double* ray_fac;   // [nlev+1] 1/(1 + dt_s tau^-1 sin^2(..)) (1 where off)
  // per-level coefficients of the column solve, colc[k*8 + j]:
  // 0 dt rd/(cvd dz_k), 1 dt (1-beta)/dz_k, 2 dt beta/dz_k, 3 dt cpd (1-beta)/dzh_k,
  // 4 dt cpd dexner_ref_ic_k, 5 dt cpd beta/dzh_k, 6 wgt_k, 7 1 - wgt_k
  const double* colc;      // [(nlev+1)*8]
};

// Work arrays of one substep / step (device, FP64).
struct DevWork {
  // edges, full levels
  double *vt, *ekin_e, *ddt_vn0, *ddt_vn1, *rho_e, *theta_e, *hpg, *vn_p;
  double *lap_vn, *nu;
  // edges, half levels
  double* gw_e;
  // cells, full levels
  double *ekin_c, *grad4, *rho_p, *exner_p, *theta_p, *divd, *div_m, *div_t, *divd2, *dtheta, *div_l, *div_vn;
  // cells, half levels
  double *ddt_w0, *ddt_w1, *w_p, *lap_w;
  // vertices
  double *zeta, *uv3, *curl_l;  // full levels (uv3: 3 fields)
  double* w_v;                  // half levels
  // column-solve scratch, level-major [k][c]
  double* col;                  // 7 planes of (nlev+1)*nc: cp, rp, rho*, pr*, rho_ic, alpha, eos
  double* zbl;                  // level-major zb [(nlev+1)*nc], predictor -> corrector
};

struct Scalars {
  double dt_s, dtime;
  double grav, rd, cpd, cvd, p00;
  double beta, wnow_vel, wnew_vel, wnow_rth, wnew_rth, exfac, divdamp, divflux;
  double rd_o_cvd, cvd_o_rd;
  int hdiff_temp;
};

// Host-side grid: validated 0-based tables plus derived factors.
struct HostGrid {
  int nc, ne, nv;
  double radius;
  std::vector<int> c2v, c2e, e2c, e2v, v2e, v2c;
  std::vector<double> cell_xyz, vert_xyz, edge_xyz;
  // derived (host copies of the device factors)
  std::vector<int> c2e2c, e2c2v, e2c2e, e2v_t;
  std::vector<double> cell_area, edge_length, dual_length, dual_area;
  std::vector<double> div_c, lap_c, e2c_w, grad_c, inv_d, inv_l, vt_w, upw, nt, inv_dn;
  std::vector<double> curl_v, c2v_w, uv_w, coriolis_z, edge_area;
  double mean_area;
};

// Builds and validates the host grid; returns an error message or "".
std::string build_host_grid(const icon_grid_desc_t* d, HostGrid* g);

}  // namespace icon
