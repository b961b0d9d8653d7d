// Internal data structures of the ICON-type dycore library (not part of the ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/icon_dycore.h"

namespace icon {

// Horizontal grid factors in device memory (row A0), in the compute type T of
// the stencil kernels (double: FP64 mode; float: mixed mode, rounded once from
// the FP64 factors).  Index tables are 0-based; pad entries of the 6-wide
// vertex tables point at a valid index and carry a zero coefficient.
template <class T>
struct GridT {
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
  const T* div_c;   // [nc*3] s_{c,e} l_e / A_c
  const T* lap_c;   // [nc*3] l_e / (d_e A_c)
  const T* e2c_w;   // [nc*3] edge->cell interpolation weights
  const T* grad_c;  // [nc*6] Green-Gauss gradient in the cell frame, (x,y) per nbr: sum G_j (psi_j - psi_c)
  const T* grad_s;  // [nc*2] sum_j G_j (x, y): the FP64 gradient as sum G_j psi_j - (sum G_j) psi_c
  const T* lap_s;   // [nc]   sum_j lap_c_j (the FP64 divergence Laplacian in the same form)
  const T* e2c_wd;  // [nc*3] e2c_w times 1/d of that edge (the sum of the edges' w advection)
  const T* k4w_c;   // [nc]   hdiff_w_k4 * A_c^2
  // edge coefficients
  const T* inv_d;   // [ne] 1/d_e
  const T* inv_l;   // [ne] 1/l_e
  const T* hinv_d;  // [ne] 1/(2 d_e) (the gradient of 2K)
  const T* d_o_l;   // [ne] d_e / l_e
  const T* f_e;     // [ne] Coriolis parameter
  const T* vt_w;    // [ne*5] tangential-wind weights: self, e2c2e[0..3]
  const T* upw;     // [ne*12] per upwind side s: (dx, dy, nx, ny, tx, ty) in that cell's frame
  const T* upw_s;   // [ne*12] the same with n and t scaled by dt_s/2 (the back trajectory's half substep)
  const T* cpd_inv_d;  // [ne] cpd / d_e (the horizontal pressure gradient's factor)
  const T* tenh_a;  // [ne] hdiff_tenh_fac A_e / dtime (enhanced temperature diffusion; null when off)
  const T* nt;      // [ne*6] normal xyz, tangent xyz
  const T* inv_dn;  // [ne] 1/(arc between the two opposite diamond vertices)
  const T* smag_a;  // [ne] hdiff_smag_fac * A_e
  const T* k4_a;    // [ne] hdiff_k4 * A_e^2
  const T* fdiv_e;  // [ne] divflux_fac * mean cell area / d_e (flux filter)
  const T* ddamp_e; // [ne] divdamp_fac * mean cell area^2 / d_e (divergence damping)
  // vertex coefficients
  const T* curl_v;  // [nv*6] t_{v,e} d_e / A_v (0 for pads)
  const T* c2v_w;   // [nv*6] cell->vertex weights (0 for pads)
  const T* uv_w;    // [nv*6*3] vertex velocity weights (xyz per edge)
  T mean_area;
  const double* cell_area;  // [nc] (diagnostics)
  const float* uv_c;        // [nc*6] east/north cell-velocity weights (corrector features)
  const float* div_c_hl;    // [nc*3*2] div_c as double-word FP32 (hi, lo) pairs (mixed flux divergence)
};
using DevGrid = GridT<double>;

// Vertical factors of the stencil kernels in the compute type T.
template <class T>
struct VertT {
  int nlev;
  const T* inv_dz;     // [nlev]
  const T* inv_dzh;    // [nlev+1]
  const T* qdz;        // [nlev] inv_dz / 4 (the vertical advection of vn: a mean of four w values)
  const T* qdzh;       // [nlev+1] inv_dzh / 2 (the vertical advection of w: a centred difference)
  const T* wgt;        // [nlev+1]
  const T* theta_ref;  // [nlev]
  const T* rho_ref;    // [nlev] (mixed mode: offset of the rho perturbation)
  const double* exner_ref;  // [nlev] (FP64 mode: exner perturbation)
};

// Terrain-following vertical coordinate (half-level heights per column): the
// per-point metrics of the stencil kernels in the compute type T, all null
// over flat ground.  Edge heights are the mean of the two cells'; slopes are
// those of the coordinate surfaces.
template <class T>
struct TerrT {
  const T* wgt_e;     // [ne*(nlev+1)] interpolation weight of level k-1 at edge half level k (0 at the ends)
  const T* qdz_e;     // [ne*nlev] 1/(4 edge layer thickness): the vertical advection's factor
  const T* ddxn_ifc;  // [ne*(nlev+1)] normal slope of the half levels, (z_c1 - z_c0)/d_e
  const T* ddxt_ifc;  // [ne*(nlev+1)] tangential slope of the half levels from the vertex heights
  const T* ddxn_mc;   // [ne*nlev] cpd times the normal slope of the full levels
  const T* qdzh_c;    // [nc*(nlev+1)] 1/(2 (z_mc[k-1] - z_mc[k])) per cell (0 at the ends)
  const T* inv_dzm_c; // [nc*nlev] 1/(z_mc[k-1] - z_mc[k+1]) per cell, one-sided at the top and the ground
  const T* fx_ratio;  // [nc*3*nlev] dz_e / dz_c of the cell's three edges (horizontal flux thickness)
  T *wcc0, *wcc1;     // work [nc*(nlev+1)]: contravariant correction of the predictor's and corrector's winds
};

// Scalars of the stencil kernels in the compute type T.
template <class T>
struct ScalT {
  T dt_s, dtime, cpd, exfac, divdamp, divflux, wnow_vel, wnew_vel;
  int hdiff_temp;
  int tenh_levels;  // enhanced temperature diffusion: the lowest levels it may act on (0: off)
  T tenh_thresh;    // its theta_v threshold, K
};

// Vertical metrics and reference state in device memory.
struct DevVert {
  int nlev;
  int n_ray;               // levels 0..n_ray-1 may be Rayleigh-damped (ray_fac 1 below, every column)
  const double* dz;        // [nlev]
  const double* inv_dz;    // [nlev]
  const double* inv_dzh;   // [nlev+1] (0 at top and ground)
  const double* wgt;       // [nlev+1] weight of level k-1 at half level k (0 at ends)
  const double* theta_ref; // [nlev]
  const double* exner_ref; // [nlev]
  const double* dexner_ref_ic;  // [nlev+1]
  const double* ray_fac;   // [nlev+1] 1/(1 + dt_s tau^-1 sin^2(..)) (1 where off)
  // per-level coefficients of the column solve, colc[k*8 + j]:
  // 0 dt rd/(cvd dz_k), 1 dt (1-beta)/dz_k, 2 dt beta/dz_k,
  // 3 theta_ref at half level k (wgt_k theta_ref_k-1 + (1 - wgt_k) theta_ref_k),
  // 4 dt cpd dexner_ref_ic_k, 5 dt cpd beta/dzh_k, 6 wgt_k, 7 1 - wgt_k
  // (3 to 7 at the interior half levels 1..nlev-1 only)
  const double* colc;      // [(nlev+1)*8]
  // the same per level as double-word FP32 pairs (hi, lo), 16 pairs per level
  // k = 0..nlev: colc 0..7, then exner_ref, theta_ref, dz, ray_fac, rho_ref
  // (zero where a quantity is not defined at that level)
  const float* lev_hl;     // [(nlev+1)*32]
  // the same 16 quantities per level in FP64, lev64[16 k + j]
  const double* lev64;     // [(nlev+1)*16]
  // terrain (null over flat ground): the reference state per column and the
  // column solve's per-level quantities per column, slot-major and level-major
  // colt[(j * (nlev+1) + k) * nc + c] (slots 0..11 as lev64; FP64 in FP64
  // mode, double-word pairs in 8-byte slots in mixed mode).  The per-level
  // tables above then hold column 0's values: the offsets of the mixed
  // mode's FP32 perturbations (any horizontally uniform profile serves).
  const double* exner_ref_c;  // [nc*nlev]
  const double* theta_ref_c;  // [nc*nlev]
  const double* dz_c;         // [nc*nlev]
  const double* colt;         // [12*(nlev+1)*nc]
  // steep terrain: the edge levels where the pressure gradient is taken at
  // constant height, steep_idx[4 i] = (edge, level, first level of the
  // quadratic in e2c[0], in e2c[1]), steep_w[6 i] = its Lagrange weights
  int n_steep;
  const int* steep_idx;
  const double* steep_w;
};

// double -> (hi, lo) FP32 pair with hi + lo = x to about 48 bits
inline void split_hl(double x, float* out) {
  const float hi = (float)x;
  out[0] = hi;
  out[1] = (float)(x - (double)hi);
}

// the lev_hl table of DevVert into t[32 (nlev + 1)] (rho_ref may be null)
inline void level_pairs_into(float* t, int nlev, const double* colc, const double* exner_ref,
                             const double* theta_ref, const double* dz, const double* ray_fac, const double* rho_ref) {
  for (size_t i = 0; i < 32 * (size_t)(nlev + 1); ++i) t[i] = 0.0f;
  for (int k = 0; k <= nlev; ++k) {
    float* r = t + 32 * (size_t)k;
    for (int j = 0; j < 8; ++j) split_hl(colc[8 * (size_t)k + j], r + 2 * j);
    if (k < nlev) {
      split_hl(exner_ref[k], r + 16);
      split_hl(theta_ref[k], r + 18);
      split_hl(dz[k], r + 20);
      if (rho_ref) split_hl(rho_ref[k], r + 24);
    }
    split_hl(ray_fac[k], r + 22);
  }
}

// the lev64 table of DevVert (the slots of lev_hl, one double each)
inline std::vector<double> level_table64(int nlev, const double* colc, const double* exner_ref, const double* theta_ref,
                                         const double* dz, const double* ray_fac, const double* rho_ref) {
  std::vector<double> t(16 * (size_t)(nlev + 1), 0.0);
  for (int k = 0; k <= nlev; ++k) {
    double* r = t.data() + 16 * (size_t)k;
    for (int j = 0; j < 8; ++j) r[j] = colc[8 * (size_t)k + j];
    if (k < nlev) {
      r[8] = exner_ref[k];
      r[9] = theta_ref[k];
      r[10] = dz[k];
      if (rho_ref) r[12] = rho_ref[k];
    }
    r[11] = ray_fac[k];
  }
  return t;
}

inline std::vector<float> level_pairs(int nlev, const double* colc, const double* exner_ref, const double* theta_ref,
                                      const double* dz, const double* ray_fac, const double* rho_ref) {
  std::vector<float> t(32 * (size_t)(nlev + 1));
  level_pairs_into(t.data(), nlev, colc, exner_ref, theta_ref, dz, ray_fac, rho_ref);
  return t;
}

// Device copy of HostVaPatches with the grid factors the fused kernel reads,
// gathered into patch order in FP32 (n_patches 0: no fused velocity advection).
// Packed tables are 16-byte aligned rows of 16-bit local indices.
struct VaPatchT {
  int P, n_patches;
  int max_e0, max_e1, max_c3, max_c0, max_v3, max_e4;
  const int *off_e0, *off_e1, *off_c0, *off_v3, *off_e4, *n_c3, *n_w4;
  const int *e0_g, *c0_g, *e4_g;
  const uint16_t *e1_i, *c3_i, *v3_i, *e4_i, *own_i;
  const float *e1_w;   // [5] per E1 item: vt_w
  const float *c3_w;   // [4] per C0 item (C3 prefix): e2c_w, 0
  const float *v3_w;   // [12] per V3 item: curl_v, c2v_w
  const float *e4_w;   // [4] per E4 item: f_e, 1/(2d), d/l, 0
  const float *own_w;  // [4] per cell: e2c_wd, 0
};

// Work arrays of the stencil kernels, compute type T.
template <class T>
struct WorkT {
  // edges, full levels
  // (ekin_e: twice the kinetic energy, vn^2 + vt^2)
  T *vt, *ekin_e, *ddt_vn0, *ddt_vn1, *rho_e, *theta_e, *hpg, *vn_p, *lap_vn, *nu;
  // edges, half levels (gw_e: the horizontal advection of w times d_e)
  T* gw_e;
  T* vn_ie;  // vn interpolated to the half levels (top: level 0, ground: level nlev-1)
  // edges, full levels (FP64 mode): the horizontal mass and theta fluxes, one value per edge
  T *flx_m, *flx_t;
  // cells, full levels (ekin_c: 2K at the cell; wq: the sum of the two w, or
  // w - w_concorr, at the level's half levels)
  T *ekin_c, *grad4, *divd, *divd2, *dtheta, *div_l, *div_vn, *wq;
  // cells, half levels
  T *ddt_w0, *ddt_w1, *lap_w;
  T* tenh_ex;  // cells, full levels: the enhanced temperature diffusion's excess factor
  // vertices
  T *zeta, *uv3, *curl_l;  // full levels (uv3: 3 fields)
  T* w_v;                  // half levels
};

// FP64 work of the column solve and the predicted state.
struct DevWork {
  double *div_m, *div_t;                  // cells: flux divergences (FP64 sums; double-word pairs in mixed mode)
  double *rho_p, *theta_p;                // cells: predicted state (the corrector's time averages)
  double* w_p;                            // cells, half levels
  double* pex;   // cells: extrapolated exner perturbation (FP64, or double-word pairs in mixed mode)
  double* col;   // level-major [k][c] scratch: 7 planes of (nlev+1)*nc: cp, rp, rho*, pr*, rho_ic, alpha, eos
  double* zbl;   // level-major zb [(nlev+1)*nc], predictor -> corrector
  double* diag;  // diagnostics: partial column-mass sums
  int* flag;     // diagnostics: non-finite flag
};

// FP32 mirrors of the state read by the mixed-mode stencils: vn, w, the
// perturbations rho - rho_ref and theta_v - theta_ref, and the predicted w.
// Written by the FP64 writers.
struct Mirrors {
  float *vn, *w, *rho, *th, *w_p;
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
  std::vector<double> curl_v, c2v_w, uv_w, coriolis_z, edge_area, uv_c;
  double mean_area;
};

// Vertical metrics, reference state, Rayleigh factors and column-solve
// coefficients of one column of half-level heights z[nlev+1] (top first).
// One routine for the flat grid and every terrain column, so that equal
// columns get bit-identical metrics.
struct ColumnMetrics {
  std::vector<double> z_mc, dz, inv_dz;      // [nlev]
  std::vector<double> inv_dzh, wgt, dref;    // [nlev+1], 0 at the top and the ground
  std::vector<double> theta_ref, exner_ref;  // [nlev]
  std::vector<double> ray;                   // [nlev+1] (1 where Rayleigh damping is off)
  std::vector<double> colc;                  // [(nlev+1)*8], layout of DevVert::colc
};
void column_metrics(const double* z, int nlev, const icon_dycore_params_t& p, const Scalars& s, ColumnMetrics* m);

// Terrain metrics on the host (see TerrT and the terrain part of DevVert).
struct HostTerrain {
  std::vector<double> exner_ref_c, theta_ref_c, dz_c, inv_dzm_c;  // [nc*nlev]
  std::vector<double> inv_dzh_c;                                  // [nc*(nlev+1)]
  std::vector<double> fx_ratio;                                   // [nc*3*nlev]
  std::vector<double> colt;                                       // [12*(nlev+1)*nc]
  std::vector<double> wgt_e, ddxn_ifc, ddxt_ifc;                  // [ne*(nlev+1)]
  std::vector<double> inv_dz_e, ddxn_mc;                          // [ne*nlev]
  std::vector<int> steep_idx;                                     // [4 n_steep] (steep_hpg)
  std::vector<double> steep_w;                                    // [6 n_steep]
  int n_ray = 0;  // the largest count of Rayleigh-damped top levels of a column
};
// Patches of the fused velocity-advection kernel (patch_setup.cpp): per
// list, the patches' entries concatenated, off_*[p] .. off_*[p+1]; C3 is the
// first n_c3[p] entries of the patch's C0 list.
struct HostVaPatches {
  int P = 0, n_patches = 0;
  int max_e0 = 0, max_e1 = 0, max_c3 = 0, max_c0 = 0, max_v3 = 0, max_e4 = 0;
  std::vector<int> off_e0, off_e1, off_c0, off_v3, off_e4, n_c3, n_w4;
  std::vector<int> e0_g;             // global edges whose vn the patch reads
  std::vector<int> e1_g, c0_g, v3_g, e4_g;
  std::vector<uint16_t> e1_i;  // [8]: local E0 of the edge and of its e2c2e, pad
  std::vector<uint16_t> c3_i;  // [4] per C0 entry: local E1 of c2e (C3 entries), pad
  std::vector<uint16_t> v3_i;  // [16]: local E0 of v2e, local C0 of v2c, pad
  std::vector<uint16_t> e4_i;  // [8]: local E1, local E0, local C0 of e2c[0], e2c[1],
                               //      local V3 of e2v[0], e2v[1], 0, 0 (the first
                               //      n_w4[p] edges are written by this patch)
  std::vector<uint16_t> own_i; // [4] per cell (global order): local E4 of c2e, 0
};
// Builds the patches of P consecutive cells; returns an error message or "".
std::string build_va_patches(const HostGrid& g, int P, HostVaPatches* out);

// Validates the per-column heights z_ifc[nc*(nlev+1)] (finite, strictly
// decreasing in every column, one common model top) and derives the terrain
// metrics; returns an error message or "".
std::string build_terrain(const HostGrid& g, int nlev, const double* z_ifc, const icon_dycore_params_t& p,
                          const Scalars& s, HostTerrain* t);

// Records `msg` as the calling thread's last error and returns `code`.
int report_error(int code, const std::string& msg);

// Builds and validates the host grid; returns an error message or "".
std::string build_host_grid(const icon_grid_desc_t* d, HostGrid* g);

}  // namespace icon
