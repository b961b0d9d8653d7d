// Row A7: vertically implicit solve of w, rho, exner and theta_v, one thread
// per column (the tridiagonal Thomas sweep is sequential in the vertical).
//
// Equations (an ICON-type reading; the paper names the solver but gives no
// formula, Sec. 4.1), for full levels k (dz) and interior half levels k (dzh),
// beta the implicit weight, pr = exner - exner_ref, primes the new values:
//   rho'_k = rho_k - dt div_m_k - dt/dz_k [(1-beta)(Fw_k - Fw_k+1) + beta(Fw'_k - Fw'_k+1)],
//   pr'_k  = pr_k - zb_k [dz_k div_t_k + (1-beta)(Gw_k - Gw_k+1) + beta(Gw'_k - Gw'_k+1)],
//   w'_k   = w_k + dt ddt_w_k - dt cpd [theta_ic ((1-beta) dpr_k + beta dpr'_k)/dzh_k
//                                       + theta'_ic dexner_ref_k],
// with Fw = rho_ic w, Gw = rho_ic theta_ic w, zb = dt (rd/cvd) exner/(rho theta dz)
// and w = 0 at the top and the ground.  Eliminating pr' gives a tridiagonal
// system in w'; Thomas elimination top-down, Rayleigh damping, then
// back-substitution; theta'_v from the linearised equation of state
//   theta' = theta (rho/rho')(1 + (cvd/rd)(pr' - pr)/exner)
//          = (dt rd/(cvd dz)) (exner - (cvd/rd) pr + (cvd/rd) pr') / (zb rho').
//
// Memory: the state is level-contiguous, so a thread walking its own column
// would read every 32-byte sector for 8 useful bytes.  Instead each CTA of
// kCW columns stages chunks of kKC levels of every input through shared
// memory with coalesced loads (a column's chunk is a contiguous run), and
// stages its outputs the same way.  The Thomas scratch is level-major
// [k][c], coalesced for one thread per column.
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels.h"

namespace icon {
namespace {

constexpr int kCW = 64;          // columns (threads) per CTA
constexpr int kKC = 8;           // levels per chunk
constexpr int kLD = kCW + 1;     // padded tile row for column-gathered tiles
constexpr int kTile = (kKC + 1) * kLD;
// forward tiles: w, rho, exner, theta, ddt_w0, div_m, div_t, ddt_w1, rho_p, theta_p, zb
constexpr int kTilesFwd = 11;
// backward: 8 level-major scratch chunks [kKC][kCW] + 4 output tiles
constexpr int kBackIn = kKC * kCW;
constexpr size_t kSmemFwd = (size_t)kTilesFwd * kTile;
constexpr size_t kSmemBack = (size_t)8 * kBackIn + 4 * (size_t)kTile;
constexpr size_t kSmem = (kSmemFwd > kSmemBack ? kSmemFwd : kSmemBack) * sizeof(double);

enum { CZB = 0, CR = 1, CRN = 2, CWX = 3, CB = 4, CGAM = 5, WG = 6, WG2 = 7 };

// Reciprocal by Newton-Raphson refinement (r <- r + r (1 - x r), quadratic
// convergence) of the hardware FP64 reciprocal approximation; two steps take
// the seed's ~20 correct bits past double precision.  Used for the pivots and
// the equation-of-state denominator, whose operands are positive and far from
// the subnormal range.
__device__ __forceinline__ double rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 8-byte asynchronous global->shared copy (no register staging), completed
// by cp_wait() for all copies the thread issued.
__device__ __forceinline__ void cp8(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) { cp8(dst, src); }
__device__ __forceinline__ void cp_async(float* dst, const float* src) { cp4(dst, src); }
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// tile[kk][col] = X[rows[col] * ld + k0 + kk] for kk < nk (level-contiguous
// field; consecutive threads copy consecutive levels of one row)
template <class T>
__device__ __forceinline__ void tile_rows(T* tile, const T* __restrict__ X, int ld, const int* __restrict__ rows,
                                          int k0, int nk) {
  for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
    const int col = i / nk, kk = i - col * nk;
    cp_async(tile + kk * kLD + col, X + (size_t)rows[col] * ld + k0 + kk);
  }
}

// tile[kk][col] = X[(k0 + kk) * nc + c0 + col] (level-major scratch), row length ldt
__device__ __forceinline__ void tile_levels(double* tile, int ldt, const double* __restrict__ X, int nc, int c0,
                                            int k0, int nk) {
  const int col = threadIdx.x;
  const int cc = c0 + col < nc ? c0 + col : nc - 1;
  for (int kk = 0; kk < nk; ++kk) cp8(tile + kk * ldt + col, X + (size_t)(k0 + kk) * nc + cc);
}

__device__ __forceinline__ void store_tile(const double* __restrict__ tile, double* X, int ld, int c0, int nc,
                                           int k0, int nk) {
  for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
    const int col = i / nk, kk = i - col * nk;
    if (c0 + col < nc) X[(size_t)(c0 + col) * ld + k0 + kk] = tile[kk * kLD + col];
  }
}

template <class T>
struct ColArgs {
  const double *w, *rho, *exner, *theta, *rho_p, *theta_p, *div_m, *div_t;
  const T *ddt_w0, *ddt_w1;
  double *zbl, *col, *w_o, *rho_o, *exner_o, *theta_o;
  // mixed mode: FP32 mirrors of the outputs (w; rho, theta_v perturbations)
  float *m_w, *m_rho, *m_th;
  const double* rho_ref;
};

template <class T>
__global__ void __launch_bounds__(kCW) sn_column_tiled(int nc, DevVert v, Scalars sc, int corrector, ColArgs<T> a) {
  extern __shared__ double sm[];
  __shared__ int rows_c[kCW];
  const int t = threadIdx.x;
  const int nlev = v.nlev, nlevp = nlev + 1;
  const int c0 = blockIdx.x * kCW;
  const int c = c0 + t;
  const bool active = c < nc;
  rows_c[t] = active ? c : nc - 1;
  __syncthreads();

  double* T_w = sm;
  double* T_rho = sm + kTile;
  double* T_pi = sm + 2 * kTile;
  double* T_th = sm + 3 * kTile;
  T* T_dw0 = reinterpret_cast<T*>(sm + 4 * kTile);
  double* T_dm = sm + 5 * kTile;
  double* T_dt = sm + 6 * kTile;
  T* T_dw1 = reinterpret_cast<T*>(sm + 7 * kTile);
  double* T_rp = sm + 8 * kTile;
  double* T_tp = sm + 9 * kTile;
  double* T_zb = sm + 10 * kTile;

  const size_t plane = (size_t)nlevp * nc;
  double* cp_s = a.col;
  double* rp_s = a.col + plane;
  double* rs_s = a.col + 2 * plane;
  double* ps_s = a.col + 3 * plane;
  double* ri_s = a.col + 4 * plane;
  double* al_s = a.col + 5 * plane;
  double* eb_s = a.col + 6 * plane;

  const double dt = sc.dt_s, beta = sc.beta, ombeta = 1.0 - beta;
  const double wn_r = sc.wnow_rth, wnew_r = sc.wnew_rth;

  // carried values: half level k (interface above full level k) and full level k-1
  double ric_k = 0.0, tic_k = 0.0, tpic_k = 0.0, rt_k = 0.0;
  double zb_km1 = 0.0, al_km1 = 0.0, ps_km1 = 0.0, pr_km1 = 0.0, cp_km1 = 0.0, rp_km1 = 0.0;

  for (int k0 = 0; k0 < nlev; k0 += kKC) {
    const int nkc = min(kKC, nlev - k0);       // levels solved in this chunk
    const int nkf = min(kKC + 1, nlev - k0);   // full levels loaded (one lookahead)
    const int nkh = min(kKC + 1, nlevp - k0);  // half levels loaded
    __syncthreads();
    tile_rows(T_w, a.w, nlevp, rows_c, k0, nkh);
    tile_rows(T_rho, a.rho, nlev, rows_c, k0, nkf);
    tile_rows(T_pi, a.exner, nlev, rows_c, k0, nkf);
    tile_rows(T_th, a.theta, nlev, rows_c, k0, nkf);
    tile_rows(T_dw0, a.ddt_w0, nlevp, rows_c, k0, nkh);
    tile_rows(T_dm, a.div_m, nlev, rows_c, k0, nkc);
    tile_rows(T_dt, a.div_t, nlev, rows_c, k0, nkc);
    if (corrector) {
      tile_rows(T_dw1, a.ddt_w1, nlevp, rows_c, k0, nkh);
      tile_rows(T_rp, a.rho_p, nlev, rows_c, k0, nkf);
      tile_rows(T_tp, a.theta_p, nlev, rows_c, k0, nkf);
      tile_levels(T_zb, kLD, a.zbl, nc, c0, k0, nkc);
    }
    cp_wait();
    __syncthreads();
    if (!active) continue;
#pragma unroll 1
    for (int kk = 0; kk < nkc; ++kk) {
      const int k = k0 + kk;
      const double* cf = v.colc + 8 * (size_t)k;
      const int o = kk * kLD + t;
      const double rho_n = T_rho[o], th_n = T_th[o], pi_n = T_pi[o];
      const double pr_k = pi_n - v.exner_ref[k];
      // interface k+1 from full levels k and k+1 (time-averaged in the corrector)
      double ric_k1 = 0.0, tic_k1 = 0.0, tpic_k1 = 0.0;
      if (k + 1 < nlev) {
        const double* cf1 = cf + 8;
        double ra = rho_n, ta = th_n, rb = T_rho[o + kLD], tb = T_th[o + kLD];
        if (corrector) {
          ra = wn_r * ra + wnew_r * T_rp[o];
          ta = wn_r * ta + wnew_r * T_tp[o];
          rb = wn_r * rb + wnew_r * T_rp[o + kLD];
          tb = wn_r * tb + wnew_r * T_tp[o + kLD];
        }
        ric_k1 = cf1[WG] * ra + cf1[WG2] * rb;
        tic_k1 = cf1[WG] * ta + cf1[WG2] * tb;
        tpic_k1 = cf1[WG] * (ta - v.theta_ref[k]) + cf1[WG2] * (tb - v.theta_ref[k + 1]);
      }
      const size_t ik = (size_t)k * nc + c;
      double zb;
      if (!corrector) {
        zb = cf[CZB] * pi_n * rcp(rho_n * th_n);
        a.zbl[ik] = zb;
        eb_s[ik] = pi_n - sc.cvd_o_rd * pr_k;
      } else {
        zb = T_zb[o];
      }
      const double wk = T_w[o], wk1 = T_w[o + kLD];
      const double rt_k1 = ric_k1 * tic_k1;
      const double rstar = rho_n - dt * T_dm[o] - cf[CR] * (ric_k * wk - ric_k1 * wk1);
      const double pstar = pr_k - zb * (v.dz[k] * T_dt[o] + ombeta * (rt_k * wk - rt_k1 * wk1));
      const double al_k = beta * rt_k, al_k1 = beta * rt_k1;
      rs_s[ik] = rstar;
      ps_s[ik] = pstar;
      ri_s[ik] = ric_k;
      al_s[ik] = al_k;
      if (k >= 1) {
        const double ddtw = corrector ? sc.wnow_vel * (double)T_dw0[o] + sc.wnew_vel * (double)T_dw1[o]
                                      : (double)T_dw0[o];
        const double wstar = wk + dt * ddtw - (cf[CWX] * tic_k * (pr_km1 - pr_k) + cf[CB] * tpic_k);
        const double gam = cf[CGAM] * tic_k;
        const double am = -gam * zb_km1 * al_km1;
        const double bm = 1.0 + gam * al_k * (zb_km1 + zb);
        const double cm = -gam * zb * al_k1;
        const double rm = wstar - gam * (ps_km1 - pstar);
        double cpk, rpk;
        if (k == 1) {
          const double inv = rcp(bm);
          cpk = cm * inv;
          rpk = rm * inv;
        } else {
          const double inv = rcp(bm - am * cp_km1);
          cpk = cm * inv;
          rpk = (rm - am * rp_km1) * inv;
        }
        cp_s[ik] = cpk;
        rp_s[ik] = rpk;
        cp_km1 = cpk;
        rp_km1 = rpk;
      }
      zb_km1 = zb;
      al_km1 = al_k;
      ps_km1 = pstar;
      pr_km1 = pr_k;
      ric_k = ric_k1;
      tic_k = tic_k1;
      tpic_k = tpic_k1;
      rt_k = rt_k1;
    }
  }

  // back-substitution, bottom to top: scratch chunks staged in, outputs staged out
  double* B_cp = sm;
  double* B_rp = sm + kBackIn;
  double* B_rs = sm + 2 * kBackIn;
  double* B_ps = sm + 3 * kBackIn;
  double* B_ri = sm + 4 * kBackIn;
  double* B_al = sm + 5 * kBackIn;
  double* B_eb = sm + 6 * kBackIn;
  double* B_zb = sm + 7 * kBackIn;
  double* O_w = sm + 8 * kBackIn;
  double* O_rho = O_w + kTile;
  double* O_pi = O_w + 2 * kTile;
  double* O_th = O_w + 3 * kTile;
  // the level-major scratch written above by this thread is read back by
  // other threads of the CTA through the asynchronous copies below
  __threadfence_block();
  double w_und_k1 = 0.0, wd_k1 = 0.0, ric_k1 = 0.0, al_k1 = 0.0;
  for (int kend = nlev; kend > 0; kend -= kKC) {
    const int k0 = max(0, kend - kKC), nk = kend - k0;
    __syncthreads();
    tile_levels(B_cp, kCW, cp_s, nc, c0, k0, nk);
    tile_levels(B_rp, kCW, rp_s, nc, c0, k0, nk);
    tile_levels(B_rs, kCW, rs_s, nc, c0, k0, nk);
    tile_levels(B_ps, kCW, ps_s, nc, c0, k0, nk);
    tile_levels(B_ri, kCW, ri_s, nc, c0, k0, nk);
    tile_levels(B_al, kCW, al_s, nc, c0, k0, nk);
    tile_levels(B_eb, kCW, eb_s, nc, c0, k0, nk);
    tile_levels(B_zb, kCW, a.zbl, nc, c0, k0, nk);
    cp_wait();
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int kk = nk - 1; kk >= 0; --kk) {
        const int k = k0 + kk;
        const double* cf = v.colc + 8 * (size_t)k;
        const int b = kk * kCW + t;
        double w_und = 0.0, wd = 0.0;
        if (k >= 1) {
          w_und = B_rp[b] - B_cp[b] * w_und_k1;
          wd = w_und * v.ray_fac[k];
        }
        const double ric = B_ri[b], al = B_al[b], zb = B_zb[b];
        const double rnew = B_rs[b] - cf[CRN] * (ric * wd - ric_k1 * wd_k1);
        const double prnew = B_ps[b] - zb * (al * wd - al_k1 * wd_k1);
        const double thnew = cf[CZB] * (B_eb[b] + sc.cvd_o_rd * prnew) * rcp(zb * rnew);
        const int o = kk * kLD + t;
        O_w[o] = wd;
        O_rho[o] = rnew;
        O_pi[o] = v.exner_ref[k] + prnew;
        O_th[o] = thnew;
        w_und_k1 = w_und;
        wd_k1 = wd;
        ric_k1 = ric;
        al_k1 = al;
      }
    }
    __syncthreads();
    store_tile(O_w, a.w_o, nlevp, c0, nc, k0, nk);
    store_tile(O_rho, a.rho_o, nlev, c0, nc, k0, nk);
    store_tile(O_pi, a.exner_o, nlev, c0, nc, k0, nk);
    store_tile(O_th, a.theta_o, nlev, c0, nc, k0, nk);
    if (a.m_w) {
      // FP32 mirrors for the mixed-mode stencils (one conversion per value)
      for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
        const int col = i / nk, kk = i - col * nk, k = k0 + kk;
        if (c0 + col >= nc) continue;
        const size_t ic = (size_t)(c0 + col) * nlev + k;
        a.m_w[(size_t)(c0 + col) * nlevp + k] = (float)O_w[kk * kLD + col];
        if (a.m_rho) {
          a.m_rho[ic] = (float)(O_rho[kk * kLD + col] - a.rho_ref[k]);
          a.m_th[ic] = (float)(O_th[kk * kLD + col] - v.theta_ref[k]);
        }
      }
    }
  }
  if (active) {
    a.w_o[(size_t)c * nlevp + nlev] = 0.0;
    if (a.m_w) a.m_w[(size_t)c * nlevp + nlev] = 0.0f;
  }
}

}  // namespace

cudaError_t init_column_kernels() {
  cudaError_t e = cudaFuncSetAttribute(sn_column_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sn_column_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

template <class T>
void launch_column(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                   cudaStream_t s) {
  const DevWork& wk = en.wk;
  ColArgs<T> a{};
  a.w = st.w;
  a.rho = st.rho;
  a.exner = st.exner;
  a.theta = st.theta_v;
  a.ddt_w0 = ddt_w0;
  a.ddt_w1 = ddt_w1;
  a.rho_p = wk.rho_p;
  a.theta_p = wk.theta_p;
  a.div_m = wk.div_m;
  a.div_t = wk.div_t;
  a.zbl = wk.zbl;
  a.col = wk.col;
  a.rho_ref = en.rho_ref64;
  const bool mixed = std::is_same<T, float>::value;
  if (corrector) {
    a.w_o = st.w;
    a.rho_o = st.rho;
    a.exner_o = st.exner;
    a.theta_o = st.theta_v;
    if (mixed) {
      a.m_w = en.m.w;
      a.m_rho = en.m.rho;
      a.m_th = en.m.th;
    }
  } else {
    a.w_o = wk.w_p;
    a.rho_o = wk.rho_p;
    a.exner_o = wk.exner_p;
    a.theta_o = wk.theta_p;
    if (mixed) a.m_w = en.m.w_p;
  }
  const unsigned blocks = (unsigned)((en.g64.nc + kCW - 1) / kCW);
  const char* name = mixed ? (corrector ? "sn_column_corr_mx" : "sn_column_pred_mx")
                           : (corrector ? "sn_column_corr" : "sn_column_pred");
  ICON_LAUNCH_SMEM(name, blocks, kCW, kSmem, s, sn_column_tiled<T>, en.g64.nc, en.v, en.sc, corrector, a);
}

template void launch_column<double>(const Engine&, int, const StateView&, const double*, const double*, cudaStream_t);
template void launch_column<float>(const Engine&, int, const StateView&, const float*, const float*, cudaStream_t);

}  // namespace icon
