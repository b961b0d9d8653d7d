// FP64 stencil kernels of one dycore step (rows A1-A10).
//
// Layout: level-contiguous X[h * nk + k] (k = 0 at the model top); one thread
// per (horizontal point, level), flattened so that the 32 lanes of a warp
// cover consecutive levels of one or two columns.  Neighbour gathers
// X[nbr * nk + k] are therefore coalesced runs of consecutive levels, and
// vertical neighbours are the adjacent words of the same run.  The column
// solve (row A7) runs one thread per column and sweeps the levels.
#include <cuda_runtime.h>

#include "kernels.h"

namespace icon {

thread_local Prof* g_prof = nullptr;

namespace {

__device__ __forceinline__ bool flat_index(int n_h, int nk, int& h, int& k) {
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n_h * (unsigned)nk) return false;
  h = (int)(i / (unsigned)nk);
  k = (int)(i - (unsigned)h * (unsigned)nk);
  return true;
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

constexpr int kThreads = 256;

// -------------------------------------------------------------------------
// A1: tangential wind and edge kinetic energy
//   vt = sum_j vt_w[j] vn[e_j] (Perot reconstruction averaged over the two
//   cells, projected on t_e), K_e = (vn^2 + vt^2)/2
// -------------------------------------------------------------------------
__global__ void va_edge_pre(DevGrid g, DevVert v, const double* __restrict__ vn,
                            double* __restrict__ vt, double* __restrict__ ekin) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const double* w = g.vt_w + 5 * (size_t)e;
  const int* q = g.e2c2e + 4 * (size_t)e;
  double vne = vn[(size_t)e * nlev + k];
  double t = w[0] * vne;
  t += w[1] * vn[(size_t)q[0] * nlev + k];
  t += w[2] * vn[(size_t)q[1] * nlev + k];
  t += w[3] * vn[(size_t)q[2] * nlev + k];
  t += w[4] * vn[(size_t)q[3] * nlev + k];
  vt[(size_t)e * nlev + k] = t;
  ekin[(size_t)e * nlev + k] = 0.5 * (vne * vne + t * t);
}

// -------------------------------------------------------------------------
// A2: cells: K_c = sum q_e K_e  (and, in the corrector, the divergence-damping
//     Laplacian dd2 = lapc(div vn*));  vertices: zeta = curl vn (full levels),
//     w_v = sum r_c w_c (half levels).  One launch over nc*nlev + nv*(nlev+1).
// -------------------------------------------------------------------------
__global__ void va_cell_vert(DevGrid g, DevVert v, const double* __restrict__ vn,
                             const double* __restrict__ w, const double* __restrict__ ekin_e,
                             double* __restrict__ ekin_c, const double* __restrict__ divd,
                             double* __restrict__ divd2, double* __restrict__ zeta,
                             double* __restrict__ w_v) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlev;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)c * nlev);
    const int* ce = g.c2e + 3 * (size_t)c;
    const double* q = g.e2c_w + 3 * (size_t)c;
    double s = q[0] * ekin_e[(size_t)ce[0] * nlev + k];
    s += q[1] * ekin_e[(size_t)ce[1] * nlev + k];
    s += q[2] * ekin_e[(size_t)ce[2] * nlev + k];
    ekin_c[i] = s;
    if (divd2) {
      const int* cc = g.c2e2c + 3 * (size_t)c;
      const double* L = g.lap_c + 3 * (size_t)c;
      double dc = divd[i];
      double r = L[0] * (divd[(size_t)cc[0] * nlev + k] - dc);
      r += L[1] * (divd[(size_t)cc[1] * nlev + k] - dc);
      r += L[2] * (divd[(size_t)cc[2] * nlev + k] - dc);
      divd2[i] = r;
    }
    return;
  }
  i -= ncell;
  if (i >= (unsigned)g.nv * nlevp) return;
  int vx = (int)(i / (unsigned)nlevp), k = (int)(i - (unsigned)vx * nlevp);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const int* vc = g.v2c + 6 * (size_t)vx;
  const double* cw = g.curl_v + 6 * (size_t)vx;
  const double* rw = g.c2v_w + 6 * (size_t)vx;
  if (k < nlev) {
    double z = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) z += cw[j] * vn[(size_t)ve[j] * nlev + k];
    zeta[(size_t)vx * nlev + k] = z;
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) s += rw[j] * w[(size_t)vc[j] * nlevp + k];
  w_v[i] = s;
}

// -------------------------------------------------------------------------
// A3: vn advective tendency (full levels) and horizontal advection of w at
//     edges (interior half levels); one launch over ne*(nlev+1).
//   ddt_vn = -(K_c1 - K_c0)/d + (zeta_e + f) vt - wbar (vn_ie_k - vn_ie_k+1)/dz
//   gw_e   = vn_ie (w_c1 - w_c0)/d + vt_ie (w_vp - w_vm)/l
// -------------------------------------------------------------------------
__global__ void va_edge_tend(DevGrid g, DevVert v, const double* __restrict__ vn,
                             const double* __restrict__ w, const double* __restrict__ vt,
                             const double* __restrict__ ekin_c, const double* __restrict__ zeta,
                             const double* __restrict__ w_v, double* __restrict__ ddt_vn,
                             double* __restrict__ gw_e) {
  int e, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.ne, nlevp, e, k)) return;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const int vm = g.e2v[2 * e], vp = g.e2v[2 * e + 1];
  const double inv_d = g.inv_d[e];
  const double* vne = vn + (size_t)e * nlev;
  const double* vte = vt + (size_t)e * nlev;
  // vn at half levels k and k+1 (top: vn_0, ground: vn_{nlev-1})
  auto vn_ie = [&](int kh) -> double {
    if (kh == 0) return vne[0];
    if (kh == nlev) return vne[nlev - 1];
    double wg = v.wgt[kh];
    return wg * vne[kh - 1] + (1.0 - wg) * vne[kh];
  };
  double vnie_k = vn_ie(k);
  if (k < nlev) {
    double vnie_k1 = vn_ie(k + 1);
    const double* w0 = w + (size_t)c0 * nlevp;
    const double* w1 = w + (size_t)c1 * nlevp;
    double wbar = 0.5 * (0.5 * (w0[k] + w0[k + 1]) + 0.5 * (w1[k] + w1[k + 1]));
    double zeta_e = 0.5 * (zeta[(size_t)vm * nlev + k] + zeta[(size_t)vp * nlev + k]);
    double dkdn = (ekin_c[(size_t)c1 * nlev + k] - ekin_c[(size_t)c0 * nlev + k]) * inv_d;
    double dvdz = (vnie_k - vnie_k1) * v.inv_dz[k];
    ddt_vn[(size_t)e * nlev + k] = -dkdn + (zeta_e + g.f_e[e]) * vte[k] - wbar * dvdz;
  }
  double gw = 0.0;
  if (k > 0 && k < nlev) {
    double wg = v.wgt[k];
    double vtie = wg * vte[k - 1] + (1.0 - wg) * vte[k];
    double dwdn = (w[(size_t)c1 * nlevp + k] - w[(size_t)c0 * nlevp + k]) * inv_d;
    double dwdt = (w_v[(size_t)vp * nlevp + k] - w_v[(size_t)vm * nlevp + k]) * g.inv_l[e];
    gw = vnie_k * dwdn + vtie * dwdt;
  }
  gw_e[(size_t)e * nlevp + k] = gw;
}

// -------------------------------------------------------------------------
// A4: w advective tendency at interior half levels (0 at top and ground)
//   ddt_w = -sum q_e gw_e - w (wf_{k-1} - wf_k)/dzh,  wf full-level averages
// -------------------------------------------------------------------------
__global__ void va_cell_w(DevGrid g, DevVert v, const double* __restrict__ w,
                          const double* __restrict__ gw_e, double* __restrict__ ddt_w) {
  int c, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.nc, nlevp, c, k)) return;
  double r = 0.0;
  if (k > 0 && k < nlev) {
    const int* ce = g.c2e + 3 * (size_t)c;
    const double* q = g.e2c_w + 3 * (size_t)c;
    double h = q[0] * gw_e[(size_t)ce[0] * nlevp + k];
    h += q[1] * gw_e[(size_t)ce[1] * nlevp + k];
    h += q[2] * gw_e[(size_t)ce[2] * nlevp + k];
    const double* wc = w + (size_t)c * nlevp;
    double wf_up = 0.5 * (wc[k - 1] + wc[k]);
    double wf_dn = 0.5 * (wc[k] + wc[k + 1]);
    r = -h - wc[k] * (wf_up - wf_dn) * v.inv_dzh[k];
  }
  ddt_w[(size_t)c * nlevp + k] = r;
}

// -------------------------------------------------------------------------
// A5 (predictor): Green-Gauss gradients of rho and theta_v in each cell's
// local frame: grad4 = (drho_x, drho_y, dth_x, dth_y) as 4 planes [4][nc*nlev].
// -------------------------------------------------------------------------
__global__ void sn_cell_grad(DevGrid g, DevVert v, const double* __restrict__ rho,
                             const double* __restrict__ theta, double* __restrict__ grad4) {
  int c, k;
  const int nlev = v.nlev;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const size_t n = (size_t)g.nc * nlev;
  const int* cc = g.c2e2c + 3 * (size_t)c;
  const double* G = g.grad_c + 8 * (size_t)c;
  size_t i = (size_t)c * nlev + k;
  size_t i0 = (size_t)cc[0] * nlev + k, i1 = (size_t)cc[1] * nlev + k, i2 = (size_t)cc[2] * nlev + k;
  double r = rho[i], r0 = rho[i0], r1 = rho[i1], r2 = rho[i2];
  double t = theta[i], t0 = theta[i0], t1 = theta[i1], t2 = theta[i2];
  grad4[i] = G[0] * r + G[2] * r0 + G[4] * r1 + G[6] * r2;
  grad4[n + i] = G[1] * r + G[3] * r0 + G[5] * r1 + G[7] * r2;
  grad4[2 * n + i] = G[0] * t + G[2] * t0 + G[4] * t1 + G[6] * t2;
  grad4[3 * n + i] = G[1] * t + G[3] * t0 + G[5] * t1 + G[7] * t2;
}

// -------------------------------------------------------------------------
// A6 (predictor edges): upwind rho_e/theta_e from the back trajectory over
// dt/2, horizontal pressure gradient with the extrapolated exner perturbation,
// and the vn predictor.
// -------------------------------------------------------------------------
__global__ void sn_edge_pred(DevGrid g, DevVert v, Scalars sc, const double* __restrict__ vn,
                             const double* __restrict__ vt, const double* __restrict__ ddt_vn,
                             const double* __restrict__ rho, const double* __restrict__ theta,
                             const double* __restrict__ exner, const double* __restrict__ exner_pr,
                             const double* __restrict__ grad4, double* __restrict__ rho_e,
                             double* __restrict__ theta_e, double* __restrict__ hpg,
                             double* __restrict__ vn_p) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t n = (size_t)g.nc * nlev;
  const size_t ie = (size_t)e * nlev + k;
  const double vne = vn[ie], vte = vt[ie];
  const int side = vne >= 0.0 ? 0 : 1;
  const int cu = g.e2c[2 * e + side];
  const double* u = g.upw + 12 * (size_t)e + 6 * side;
  const double hdt = 0.5 * sc.dt_s;
  double dx = u[0] - hdt * (vne * u[2] + vte * u[4]);
  double dy = u[1] - hdt * (vne * u[3] + vte * u[5]);
  size_t iu = (size_t)cu * nlev + k;
  double re = rho[iu] + (grad4[iu] * dx + grad4[n + iu] * dy);
  double te = theta[iu] + (grad4[2 * n + iu] * dx + grad4[3 * n + iu] * dy);
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const double pref = v.exner_ref[k];
  const size_t i0 = (size_t)c0 * nlev + k, i1 = (size_t)c1 * nlev + k;
  double pex0 = (1.0 + sc.exfac) * (exner[i0] - pref) - sc.exfac * exner_pr[i0];
  double pex1 = (1.0 + sc.exfac) * (exner[i1] - pref) - sc.exfac * exner_pr[i1];
  double h = sc.cpd * te * ((pex1 - pex0) * g.inv_d[e]);
  double vnp = vne + sc.dt_s * (ddt_vn[ie] - h);
  rho_e[ie] = re;
  theta_e[ie] = te;
  hpg[ie] = h;
  vn_p[ie] = vnp;
}

// -------------------------------------------------------------------------
// A8 + A9 (corrector edges): vn corrector with time-weighted advective
// tendencies, the predictor's pressure gradient and fourth-order divergence
// damping.  vn is updated in place.
// -------------------------------------------------------------------------
__global__ void sn_edge_corr(DevGrid g, DevVert v, Scalars sc, double* __restrict__ vn,
                             const double* __restrict__ ddt_vn0, const double* __restrict__ ddt_vn1,
                             const double* __restrict__ hpg, const double* __restrict__ divd2) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t ie = (size_t)e * nlev + k;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const double dd = (divd2[(size_t)c1 * nlev + k] - divd2[(size_t)c0 * nlev + k]) * g.inv_d[e];
  const double am = g.mean_area;
  double vnn = vn[ie] + sc.dt_s * (sc.wnow_vel * ddt_vn0[ie] + sc.wnew_vel * ddt_vn1[ie] - hpg[ie]) -
               sc.divdamp * am * am * dd;
  vn[ie] = vnn;
}

// -------------------------------------------------------------------------
// Cell divergence of an edge field, D = (1/A_c) sum_e s l_e vn_e: the
// divergence of vn* (fourth-order damping and flux filter of the predictor)
// or of vn^{n+1} (flux filter of the corrector).
// -------------------------------------------------------------------------
// In the predictor launch it also updates the exner extrapolation history,
// exner_pr = exner - exner_ref (sn_edge_pred, the last reader of the old
// history, has completed).
__global__ void sn_cell_div(DevGrid g, DevVert v, const double* __restrict__ vn, double* __restrict__ divd,
                            const double* __restrict__ exner, double* __restrict__ exner_pr) {
  int c, k;
  const int nlev = v.nlev;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const int* ce = g.c2e + 3 * (size_t)c;
  const double* dv = g.div_c + 3 * (size_t)c;
  const size_t i = (size_t)c * nlev + k;
  divd[i] = dv[0] * vn[(size_t)ce[0] * nlev + k] + dv[1] * vn[(size_t)ce[1] * nlev + k] +
            dv[2] * vn[(size_t)ce[2] * nlev + k];
  if (exner_pr) exner_pr[i] = exner[i] - v.exner_ref[k];
}

// -------------------------------------------------------------------------
// Divergences of the horizontal mass and theta fluxes with the flux-velocity
// filter, per cell and level:
//   vf_e = vn_e + divflux (D_c1 - D_c0)/d_e,  F_e = rho_e vf_e,
//   div_m = sum s l F / A,  div_t = sum s l F theta_e / A
// -------------------------------------------------------------------------
__global__ void sn_cell_fluxdiv(DevGrid g, DevVert v, Scalars sc, const double* __restrict__ vn,
                                const double* __restrict__ divd, const double* __restrict__ rho_e,
                                const double* __restrict__ theta_e, double* __restrict__ div_m,
                                double* __restrict__ div_t) {
  int c, k;
  const int nlev = v.nlev;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const int* ce = g.c2e + 3 * (size_t)c;
  const double* dv = g.div_c + 3 * (size_t)c;
  double dm = 0.0, dt = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int e = ce[j];
    const size_t ie = (size_t)e * nlev + k;
    const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
    const double vf = vn[ie] + sc.divflux * g.inv_d[e] * (divd[(size_t)c1 * nlev + k] - divd[(size_t)c0 * nlev + k]);
    const double f = rho_e[ie] * vf;
    dm += dv[j] * f;
    dt += dv[j] * (f * theta_e[ie]);
  }
  div_m[(size_t)c * nlev + k] = dm;
  div_t[(size_t)c * nlev + k] = dt;
}

// -------------------------------------------------------------------------
// A10 diffusion
// -------------------------------------------------------------------------
// cells: div vn; vertices: curl vn and the vertex velocity (xyz)
__global__ void diff_div_curl_uv(DevGrid g, DevVert v, const double* __restrict__ vn,
                                 double* __restrict__ div_vn, double* __restrict__ zeta,
                                 double* __restrict__ uv3) {
  const int nlev = v.nlev;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlev;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)c * nlev);
    const int* ce = g.c2e + 3 * (size_t)c;
    const double* dv = g.div_c + 3 * (size_t)c;
    div_vn[i] = dv[0] * vn[(size_t)ce[0] * nlev + k] + dv[1] * vn[(size_t)ce[1] * nlev + k] +
                dv[2] * vn[(size_t)ce[2] * nlev + k];
    return;
  }
  i -= ncell;
  const size_t nvl = (size_t)g.nv * nlev;
  if (i >= nvl) return;
  int vx = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)vx * nlev);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const double* cw = g.curl_v + 6 * (size_t)vx;
  const double* U = g.uv_w + 18 * (size_t)vx;
  double z = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double x = vn[(size_t)ve[j] * nlev + k];
    z += cw[j] * x;
    ux += U[3 * j] * x;
    uy += U[3 * j + 1] * x;
    uz += U[3 * j + 2] * x;
  }
  zeta[i] = z;
  uv3[i] = ux;
  uv3[nvl + i] = uy;
  uv3[2 * nvl + i] = uz;
}

// edges: Smagorinsky coefficient and the vector Laplacian of vn
__global__ void diff_edge_smag(DevGrid g, DevVert v, const double* __restrict__ div_vn,
                               const double* __restrict__ zeta, const double* __restrict__ uv3,
                               double* __restrict__ nu, double* __restrict__ lap) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t nvl = (size_t)g.nv * nlev;
  const int* dm = g.e2c2v + 4 * (size_t)e;
  const size_t im = (size_t)dm[0] * nlev + k, ip = (size_t)dm[1] * nlev + k;
  const size_t i2 = (size_t)dm[2] * nlev + k, i3 = (size_t)dm[3] * nlev + k;
  const double* nt = g.nt + 6 * (size_t)e;
  double dtx = uv3[ip] - uv3[im], dty = uv3[nvl + ip] - uv3[nvl + im], dtz = uv3[2 * nvl + ip] - uv3[2 * nvl + im];
  double dnx = uv3[i3] - uv3[i2], dny = uv3[nvl + i3] - uv3[nvl + i2], dnz = uv3[2 * nvl + i3] - uv3[2 * nvl + i2];
  const double il = g.inv_l[e], idn = g.inv_dn[e];
  double tension = (dnx * nt[0] + dny * nt[1] + dnz * nt[2]) * idn - (dtx * nt[3] + dty * nt[4] + dtz * nt[5]) * il;
  double shear = (dtx * nt[0] + dty * nt[1] + dtz * nt[2]) * il + (dnx * nt[3] + dny * nt[4] + dnz * nt[5]) * idn;
  const size_t ie = (size_t)e * nlev + k;
  nu[ie] = g.smag_a[e] * sqrt(tension * tension + shear * shear);
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  lap[ie] = (div_vn[(size_t)c1 * nlev + k] - div_vn[(size_t)c0 * nlev + k]) * g.inv_d[e] -
            (zeta[ip] - zeta[im]) * il;
}

// cells (half-level range): div of lap vn, cell Laplacian of w, theta increment;
// vertices: curl of lap vn
__global__ void diff_second(DevGrid g, DevVert v, Scalars sc, const double* __restrict__ lap,
                            const double* __restrict__ nu, const double* __restrict__ w,
                            const double* __restrict__ theta, double* __restrict__ div_l,
                            double* __restrict__ lap_w, double* __restrict__ dtheta,
                            double* __restrict__ curl_l) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlevp;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlevp), k = (int)(i - (unsigned)c * nlevp);
    const int* ce = g.c2e + 3 * (size_t)c;
    const int* cc = g.c2e2c + 3 * (size_t)c;
    const double* L = g.lap_c + 3 * (size_t)c;
    const double wc = w[(size_t)c * nlevp + k];
    double lw = L[0] * (w[(size_t)cc[0] * nlevp + k] - wc);
    lw += L[1] * (w[(size_t)cc[1] * nlevp + k] - wc);
    lw += L[2] * (w[(size_t)cc[2] * nlevp + k] - wc);
    lap_w[i] = lw;
    if (k < nlev) {
      const double* dv = g.div_c + 3 * (size_t)c;
      const size_t ic = (size_t)c * nlev + k;
      div_l[ic] = dv[0] * lap[(size_t)ce[0] * nlev + k] + dv[1] * lap[(size_t)ce[1] * nlev + k] +
                  dv[2] * lap[(size_t)ce[2] * nlev + k];
      if (sc.hdiff_temp) {
        const double tc = theta[ic];
        double f = L[0] * nu[(size_t)ce[0] * nlev + k] * (theta[(size_t)cc[0] * nlev + k] - tc);
        f += L[1] * nu[(size_t)ce[1] * nlev + k] * (theta[(size_t)cc[1] * nlev + k] - tc);
        f += L[2] * nu[(size_t)ce[2] * nlev + k] * (theta[(size_t)cc[2] * nlev + k] - tc);
        dtheta[ic] = sc.dtime * f;
      }
    }
    return;
  }
  i -= ncell;
  if (i >= (unsigned)g.nv * nlev) return;
  int vx = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)vx * nlev);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const double* cw = g.curl_v + 6 * (size_t)vx;
  double z = 0.0;
#pragma unroll
  for (int j = 0; j < 6; ++j) z += cw[j] * lap[(size_t)ve[j] * nlev + k];
  curl_l[i] = z;
}

// edges: vn update (in place)
__global__ void diff_edge_update(DevGrid g, DevVert v, Scalars sc, double* __restrict__ vn,
                                 const double* __restrict__ nu, const double* __restrict__ lap,
                                 const double* __restrict__ div_l, const double* __restrict__ curl_l) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t ie = (size_t)e * nlev + k;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const int vm = g.e2v[2 * e], vp = g.e2v[2 * e + 1];
  double lap2 = (div_l[(size_t)c1 * nlev + k] - div_l[(size_t)c0 * nlev + k]) * g.inv_d[e] -
                (curl_l[(size_t)vp * nlev + k] - curl_l[(size_t)vm * nlev + k]) * g.inv_l[e];
  vn[ie] = vn[ie] + sc.dtime * nu[ie] * lap[ie] - g.k4_a[e] * lap2;
}

// cells (half-level range): w fourth-order diffusion, theta/exner update (in place)
__global__ void diff_cell_update(DevGrid g, DevVert v, Scalars sc, double* __restrict__ w,
                                 double* __restrict__ theta, double* __restrict__ exner,
                                 const double* __restrict__ lap_w, const double* __restrict__ dtheta) {
  int c, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.nc, nlevp, c, k)) return;
  if (k > 0 && k < nlev) {
    const int* cc = g.c2e2c + 3 * (size_t)c;
    const double* L = g.lap_c + 3 * (size_t)c;
    const double lc = lap_w[(size_t)c * nlevp + k];
    double l2 = L[0] * (lap_w[(size_t)cc[0] * nlevp + k] - lc);
    l2 += L[1] * (lap_w[(size_t)cc[1] * nlevp + k] - lc);
    l2 += L[2] * (lap_w[(size_t)cc[2] * nlevp + k] - lc);
    w[(size_t)c * nlevp + k] -= g.k4w_c[c] * l2;
  }
  if (k < nlev && sc.hdiff_temp) {
    const size_t ic = (size_t)c * nlev + k;
    const double th = theta[ic];
    const double thn = th + dtheta[ic];
    theta[ic] = thn;
    exner[ic] = exner[ic] * (1.0 + sc.rd_o_cvd * (thn - th) / th);
  }
}

}  // namespace

// -------------------------------------------------------------------------
// launch wrappers
// -------------------------------------------------------------------------
void launch_velocity_tendencies(const DevGrid& g, const DevVert& v, const double* vn, const double* w,
                                DevWork& wk, double* ddt_vn, double* ddt_w, const double* divd,
                                double* divd2, cudaStream_t s) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  ICON_LAUNCH("va_edge_pre", blocks_for((long long)g.ne * nlev, kThreads), kThreads, s, va_edge_pre, g, v, vn, wk.vt, wk.ekin_e);
  long long n2 = (long long)g.nc * nlev + (long long)g.nv * nlevp;
  ICON_LAUNCH("va_cell_vert", blocks_for(n2, kThreads), kThreads, s, va_cell_vert, g, v, vn, w, wk.ekin_e, wk.ekin_c, divd, divd2,
                                                              wk.zeta, wk.w_v);
  ICON_LAUNCH("va_edge_tend", blocks_for((long long)g.ne * nlevp, kThreads), kThreads, s, va_edge_tend, 
      g, v, vn, w, wk.vt, wk.ekin_c, wk.zeta, wk.w_v, ddt_vn, wk.gw_e);
  ICON_LAUNCH("va_cell_w", blocks_for((long long)g.nc * nlevp, kThreads), kThreads, s, va_cell_w, g, v, w, wk.gw_e, ddt_w);
}

void launch_substep(const DevGrid& g, const DevVert& v, const Scalars& sc, const StateView& st, DevWork& wk,
                    cudaStream_t s) {
  const int nlev = v.nlev;
  const unsigned bc = blocks_for((long long)g.nc * nlev, kThreads), be = blocks_for((long long)g.ne * nlev, kThreads);
  // ---------------- predictor ----------------
  launch_velocity_tendencies(g, v, st.vn, st.w, wk, wk.ddt_vn0, wk.ddt_w0, nullptr, nullptr, s);
  ICON_LAUNCH("sn_cell_grad", bc, kThreads, s, sn_cell_grad, g, v, st.rho, st.theta_v, wk.grad4);
  ICON_LAUNCH("sn_edge_pred", be, kThreads, s, sn_edge_pred, g, v, sc, st.vn, wk.vt, wk.ddt_vn0, st.rho, st.theta_v,
              st.exner, st.exner_pr, wk.grad4, wk.rho_e, wk.theta_e, wk.hpg, wk.vn_p);
  ICON_LAUNCH("sn_cell_div", bc, kThreads, s, sn_cell_div, g, v, wk.vn_p, wk.divd, st.exner, st.exner_pr);
  ICON_LAUNCH("sn_cell_fluxdiv", bc, kThreads, s, sn_cell_fluxdiv, g, v, sc, wk.vn_p, wk.divd, wk.rho_e, wk.theta_e,
              wk.div_m, wk.div_t);
  launch_column(g, v, sc, 0, st, wk, s);
  // ---------------- corrector ----------------
  launch_velocity_tendencies(g, v, wk.vn_p, wk.w_p, wk, wk.ddt_vn1, wk.ddt_w1, wk.divd, wk.divd2, s);
  ICON_LAUNCH("sn_edge_corr", be, kThreads, s, sn_edge_corr, g, v, sc, st.vn, wk.ddt_vn0, wk.ddt_vn1, wk.hpg,
              wk.divd2);
  ICON_LAUNCH("sn_cell_div", bc, kThreads, s, sn_cell_div, g, v, st.vn, wk.divd, nullptr, nullptr);
  ICON_LAUNCH("sn_cell_fluxdiv", bc, kThreads, s, sn_cell_fluxdiv, g, v, sc, st.vn, wk.divd, wk.rho_e, wk.theta_e,
              wk.div_m, wk.div_t);
  launch_column(g, v, sc, 1, st, wk, s);
}

void launch_diffusion(const DevGrid& g, const DevVert& v, const Scalars& sc, const StateView& st, DevWork& wk,
                      cudaStream_t s) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  long long n1 = (long long)g.nc * nlev + (long long)g.nv * nlev;
  ICON_LAUNCH("diff_div_curl_uv", blocks_for(n1, kThreads), kThreads, s, diff_div_curl_uv, g, v, st.vn, wk.div_vn, wk.zeta, wk.uv3);
  ICON_LAUNCH("diff_edge_smag", blocks_for((long long)g.ne * nlev, kThreads), kThreads, s, diff_edge_smag, g, v, wk.div_vn, wk.zeta,
                                                                                    wk.uv3, wk.nu, wk.lap_vn);
  long long n3 = (long long)g.nc * nlevp + (long long)g.nv * nlev;
  ICON_LAUNCH("diff_second", blocks_for(n3, kThreads), kThreads, s, diff_second, g, v, sc, wk.lap_vn, wk.nu, st.w, st.theta_v,
                                                             wk.div_l, wk.lap_w, wk.dtheta, wk.curl_l);
  ICON_LAUNCH("diff_edge_update", blocks_for((long long)g.ne * nlev, kThreads), kThreads, s, diff_edge_update, g, v, sc, st.vn, wk.nu,
                                                                                      wk.lap_vn, wk.div_l,
                                                                                      wk.curl_l);
  ICON_LAUNCH("diff_cell_update", blocks_for((long long)g.nc * nlevp, kThreads), kThreads, s, diff_cell_update, g, v, sc, st.w,
                                                                                       st.theta_v, st.exner,
                                                                                       wk.lap_w, wk.dtheta);
}

}  // namespace icon
