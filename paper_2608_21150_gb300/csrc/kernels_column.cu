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
// kCW columns stages chunks of KC levels (4, 6 or 8, picked by the
// autotuner) of every input through shared memory with coalesced loads (a
// column's chunk is a contiguous run), and stages its outputs the same way.
// The Thomas scratch is level-major
// [k][c], coalesced for one thread per column; it is written as streaming
// data and read back evict-first, while the input rows are kept (L2 policies
// below).  Each chunk's slice of the per-level table is staged in shared
// memory as well (FP64 or double-word): every thread of the CTA reads the same
// level at the same time, and from L1 those loads were a large share of the
// kernel's stalls.  The predictor and corrector forms are separate kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>

#include "dfloat.cuh"
#include "kernels.h"

namespace icon {
namespace {

constexpr int kCW = 64;          // columns (threads) per CTA
constexpr int kKC = 4;           // default levels per chunk (the autotuner picks 4, 6 or 8)
constexpr int kLD = kCW + 1;     // padded tile row for column-gathered tiles
template <int KC>
__host__ __device__ constexpr int tile_doubles() { return (KC + 1) * kLD; }
// Shared memory of one CTA, in bytes.  Forward: the FP64 tiles w, rho,
// exner, theta, div_m, div_t (+ rho_p, theta_p, zb in the corrector), then
// the tendency tiles ddt_w0 (+ ddt_w1) of the stencils' type T, each
// (KC + 1) x kLD.  Backward (reusing it): 8 level-major scratch chunks
// [KC][kCW] and 4 output tiles [KC][kLD].  Then the per-level table of a
// chunk: 16 slots per level, KC + 1 levels.  kCorrTiles: room for the
// corrector's tiles.
template <class T, int KC, bool kCorrTiles>
__host__ __device__ constexpr int fwd_bytes() {
  return (6 + (kCorrTiles ? 3 : 0)) * tile_doubles<KC>() * 8 + (kCorrTiles ? 2 : 1) * tile_doubles<KC>() * (int)sizeof(T);
}
template <int KC>
__host__ __device__ constexpr int back_bytes() {
  return (8 * KC * kCW + 4 * KC * kLD) * 8;
}
template <class T, int KC, bool kCorrTiles>
__host__ __device__ constexpr int lev_offset_bytes() {
  return ((fwd_bytes<T, KC, kCorrTiles>() > back_bytes<KC>() ? fwd_bytes<T, KC, kCorrTiles>() : back_bytes<KC>()) +
          15) /
         16 * 16;
}
template <class T, int KC, bool kCorrTiles>
constexpr size_t smem_bytes() {
  return (size_t)lev_offset_bytes<T, KC, kCorrTiles>() + 16 * (size_t)(KC + 1) * sizeof(double);
}
constexpr size_t kSmem = smem_bytes<double, kKC, true>();

enum { CZB = 0, CR = 1, CRN = 2, CWX = 3, CB = 4, CGAM = 5, WG = 6, WG2 = 7 };

// Reciprocal of a positive FP64 value far from the subnormal range (the
// pivots and the equation-of-state denominator): a double-word FP32 seed
// (about 44 correct bits, computed on the FP32 pipes) widened with one FP64
// addition, then one Newton-Raphson step r + r (1 - x r) in FP64, which
// squares the seed's relative error to far below double precision.  Three
// operations on this GPU's slow FP64 pipe instead of the five of the
// hardware approximation refined twice.
__device__ __forceinline__ double rcp(double x) {
  const double r = to_double(icon::rcp(to_df(x)));
  const double e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 8-byte asynchronous global->shared copy (no register staging), completed
// by cp_wait() for all copies the thread issued.
__device__ __forceinline__ void cp8(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
// The row-gathered input copies mark their lines evict-last in L2: a chunk
// reads a few levels of every row, so the rest of a 128-byte line is used
// by the next chunks of the same CTA, and the Thomas scratch streaming
// through L2 meanwhile should be evicted first.
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile(
      "{\n.reg .b64 pol;\ncreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n"
      "cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, pol;\n}\n" ::"r"(s),
      "l"(src)
      : "memory");
}
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile(
      "{\n.reg .b64 pol;\ncreatepolicy.fractional.L2::evict_last.b64 pol, 1.0;\n"
      "cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, pol;\n}\n" ::"r"(s),
      "l"(src)
      : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// tile[kk][col] = X[rows[col] * ld + k0 + kk] for kk < nk (level-contiguous
// field; consecutive threads copy consecutive levels of one row).  Each of the
// kCW threads makes exactly nk copies; with nk a compile-time constant (the
// full chunks) the index split needs no run-time division.
template <int NK, class T>
__device__ __forceinline__ void tile_rows_n(T* tile, const T* __restrict__ X, int ld, const int* __restrict__ rows,
                                            int k0) {
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const int i = threadIdx.x + j * kCW;
    const int col = i / NK, kk = i - col * NK;
    cp_async(tile + kk * kLD + col, X + (size_t)rows[col] * ld + k0 + kk);
  }
}
template <int KC, class T>
__device__ __forceinline__ void tile_rows(T* tile, const T* __restrict__ X, int ld, const int* __restrict__ rows,
                                          int k0, int nk) {
  if (nk == KC + 1) {
    tile_rows_n<KC + 1>(tile, X, ld, rows, k0);
  } else if (nk == KC) {
    tile_rows_n<KC>(tile, X, ld, rows, k0);
  } else {
    for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
      const int col = i / nk, kk = i - col * nk;
      cp_async(tile + kk * kLD + col, X + (size_t)rows[col] * ld + k0 + kk);
    }
  }
}

// tile[kk][col] = X[(k0 + kk) * nc + c0 + col] (level-major scratch), row length ldt
__device__ __forceinline__ void tile_levels(double* tile, int ldt, const double* __restrict__ X, int nc, int c0,
                                            int k0, int nk) {
  const int col = threadIdx.x;
  const int cc = c0 + col < nc ? c0 + col : nc - 1;
  for (int kk = 0; kk < nk; ++kk) cp8(tile + kk * ldt + col, X + (size_t)(k0 + kk) * nc + cc);
}

// L2 policy for data read for the last time: its lines are the first to go,
// so that the partly consumed input rows of the forward sweep stay resident
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}

// tile_levels for scratch read for the last time (evict-first in L2)
__device__ __forceinline__ void tile_levels_last(double* tile, int ldt, const double* __restrict__ X, int nc, int c0,
                                                 int k0, int nk, unsigned long long pol) {
  const int col = threadIdx.x;
  const int cc = c0 + col < nc ? c0 + col : nc - 1;
  const unsigned s = (unsigned)__cvta_generic_to_shared(tile + col);
  for (int kk = 0; kk < nk; ++kk)
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s + kk * ldt * 8),
                 "l"(X + (size_t)(k0 + kk) * nc + cc), "l"(pol)
                 : "memory");
}

template <int NK>
__device__ __forceinline__ void store_tile_n(const double* __restrict__ tile, double* X, int ld, int c0, int nc,
                                             int k0) {
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const int i = threadIdx.x + j * kCW;
    const int col = i / NK, kk = i - col * NK;
    if (c0 + col < nc) X[(size_t)(c0 + col) * ld + k0 + kk] = tile[kk * kLD + col];
  }
}
template <int KC>
__device__ __forceinline__ void store_tile(const double* __restrict__ tile, double* X, int ld, int c0, int nc,
                                           int k0, int nk) {
  if (nk == KC) {
    store_tile_n<KC>(tile, X, ld, c0, nc, k0);
  } else {
    for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
      const int col = i / nk, kk = i - col * nk;
      if (c0 + col < nc) X[(size_t)(c0 + col) * ld + k0 + kk] = tile[kk * kLD + col];
    }
  }
}

// FP32 mirrors of a finished chunk (mixed mode), from the float pairs the
// back-substitution left in its consumed scratch slots: (w, rho - rho_ref) in
// m01[kk][col], theta_v - theta_ref in m2[kk][col]
template <int NK>
__device__ __forceinline__ void mirror_chunk_n(const double* m01, const double* m2, float* m_w, float* m_rho,
                                               float* m_th, int nlev, int c0, int nc, int k0) {
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const int i = threadIdx.x + j * kCW;
    const int col = i / NK, kk = i - col * NK, k = k0 + kk;
    if (c0 + col >= nc) continue;
    const float* m = reinterpret_cast<const float*>(m01 + kk * kCW + col);
    m_w[(size_t)(c0 + col) * (nlev + 1) + k] = m[0];
    if (m_rho) {
      const size_t ic = (size_t)(c0 + col) * nlev + k;
      m_rho[ic] = m[1];
      m_th[ic] = reinterpret_cast<const float*>(m2 + kk * kCW + col)[0];
    }
  }
}
template <int KC>
__device__ __forceinline__ void mirror_chunk(const double* m01, const double* m2, float* m_w, float* m_rho,
                                             float* m_th, int nlev, int c0, int nc, int k0, int nk) {
  if (nk == KC) {
    mirror_chunk_n<KC>(m01, m2, m_w, m_rho, m_th, nlev, c0, nc, k0);
  } else {
    for (int i = threadIdx.x; i < nk * kCW; i += kCW) {
      const int col = i / nk, kk = i - col * nk, k = k0 + kk;
      if (c0 + col >= nc) continue;
      const float* m = reinterpret_cast<const float*>(m01 + kk * kCW + col);
      m_w[(size_t)(c0 + col) * (nlev + 1) + k] = m[0];
      if (m_rho) {
        const size_t ic = (size_t)(c0 + col) * nlev + k;
        m_rho[ic] = m[1];
        m_th[ic] = reinterpret_cast<const float*>(m2 + kk * kCW + col)[0];
      }
    }
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

// Arithmetic of the solve: FP64 (R = double), or double-word FP32 (R = dws,
// mixed precision) with inputs split and outputs joined at the tile boundary.
template <class R>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double in(double x) { return x; }
  static __device__ __forceinline__ double in(float x) { return (double)x; }
  static __device__ __forceinline__ double inv(double x) { return rcp(x); }
  static __device__ __forceinline__ double out(double x) { return x; }
};
template <>
struct Ar<dws> {
  static __device__ __forceinline__ dws in(double x) { return to_dws(to_df(x)); }
  static __device__ __forceinline__ dws in(float x) { return {x, 0.0f}; }
  static __device__ __forceinline__ dws inv(dws x) { return rcp(x); }
  static __device__ __forceinline__ double out(dws x) { return to_double(x); }
};

// per-level quantities: j < 8 the column coefficients, then these
enum { LEX = 8, LTH = 9, LDZ = 10, LRAY = 11, LRHO = 12 };
template <class R, int J>
__device__ __forceinline__ R lev(const DevVert& v, int k);
template <>
__device__ __forceinline__ double lev<double, LEX>(const DevVert& v, int k) { return v.exner_ref[k]; }
template <>
__device__ __forceinline__ double lev<double, LTH>(const DevVert& v, int k) { return v.theta_ref[k]; }
template <>
__device__ __forceinline__ double lev<double, LDZ>(const DevVert& v, int k) { return v.dz[k]; }
template <>
__device__ __forceinline__ double lev<double, LRAY>(const DevVert& v, int k) { return v.ray_fac[k]; }
template <class R, int J>
__device__ __forceinline__ R lev(const DevVert& v, int k) {
  if constexpr (!std::is_same<R, double>::value) {
    return reinterpret_cast<const R*>(v.lev_hl)[16 * (size_t)k + J];
  } else {
    static_assert(J < 8, "column coefficient");
    return v.colc[8 * (size_t)k + J];
  }
}

// Per-level quantity of level k: from the chunk's copy of the table in shared
// memory (Ls: levels from k0 on, 16 slots each; kStaged), else from the
// device arrays.
template <class R, int J, bool kStaged>
__device__ __forceinline__ R levs(const DevVert& v, const double* Ls, int k, int k0) {
  if constexpr (kStaged) {
    return *reinterpret_cast<const R*>(Ls + 16 * (k - k0) + J);
  } else {
    return lev<R, J>(v, k);
  }
}

// A value the mixed-precision step (T = float) keeps as a double-word pair in
// an 8-byte slot -- the flux divergences and the predictor's rho and theta_v
// -- read as the pair; otherwise an FP64 value, converted.
template <class T, class R>
__device__ __forceinline__ R stored_in(const double* p) {
  if constexpr (std::is_same<T, float>::value && !std::is_same<R, double>::value) {
    return *reinterpret_cast<const R*>(p);
  } else {
    return Ar<R>::in(*p);
  }
}

// Sum of two non-negative values (densities, potential temperatures, positive
// coefficients): the cheaper double-word addition is exact enough without
// cancellation; plain addition in FP64.
__device__ __forceinline__ double add_pos(double a, double b) { return a + b; }
__device__ __forceinline__ dws add_pos(dws a, dws b) { return a + b; }

// Scratch planes hold R values in 8-byte slots (a double-word value is two floats).  They
// are read back only after the whole forward sweep, so they are stored as
// streaming (evict-first) data that does not displace the input rows in L2.
__device__ __forceinline__ void put(double* p, double x) { __stcs(p, x); }
__device__ __forceinline__ void put(double* p, dws x) { __stcs(reinterpret_cast<float2*>(p), make_float2(x.hi, x.lo)); }
template <class R>
__device__ __forceinline__ R get(const double* p) {
  return *reinterpret_cast<const R*>(p);
}

// kOwnZb: the corrector form computes zb and the equation-of-state term itself
// (as the predictor does) instead of reading the predictor's; used by the
// allocation-free entry point below.
// kCorr: 0 the predictor form, 1 the corrector form, -1 the form the
// `corrector` argument names (one kernel for both; the allocation-free entry).
// The fixed forms are separate, smaller kernels.
template <class T, bool kOwnZb = false, int KC = kKC, class R = double, int kCorr = -1>
__global__ void __launch_bounds__(kCW, 8) sn_column_tiled(int nc, DevVert v, Scalars sc, int corrector_arg,
                                                          ColArgs<T> a) {
  const bool corrector = kCorr < 0 ? corrector_arg != 0 : kCorr == 1;
  using A = Ar<R>;
  constexpr bool kDW = !std::is_same<R, double>::value;
  // the mixed step's engine path (FP32 stencil inputs, double-word solve)
  constexpr bool kPairs = std::is_same<T, float>::value && kDW;
  constexpr int kTile = tile_doubles<KC>();
  constexpr int kBackIn = KC * kCW;
  constexpr int kOut = KC * kLD;
  constexpr bool kCT = kCorr != 0;
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
  double* T_dm = sm + 4 * kTile;
  double* T_dt = sm + 5 * kTile;
  double* T_rp = sm + 6 * kTile;  // corrector tiles (kCT)
  double* T_tp = sm + 7 * kTile;
  double* T_zb = sm + 8 * kTile;
  T* T_dw0 = reinterpret_cast<T*>(sm + (kCT ? 9 : 6) * kTile);
  T* T_dw1 = T_dw0 + kTile;
  // the per-level table is staged per chunk, except in the FP64 form of the
  // allocation-free entry, which has no FP64 copy of the table
  constexpr bool kStage = kDW || !kOwnZb;
  double* L_s = sm + lev_offset_bytes<T, KC, kCT>() / 8;
  const double* lev_src = kDW ? reinterpret_cast<const double*>(v.lev_hl) : v.lev64;

  const size_t plane = (size_t)nlevp * nc;
  double* cp_s = a.col;
  double* rp_s = a.col + plane;
  double* rs_s = a.col + 2 * plane;
  double* ps_s = a.col + 3 * plane;
  double* ri_s = a.col + 4 * plane;
  double* al_s = a.col + 5 * plane;
  double* eb_s = a.col + 6 * plane;

  const R zero = A::in(0.0), one = A::in(1.0);
  const R dt = A::in(sc.dt_s), beta = A::in(sc.beta), ombeta = A::in(1.0 - sc.beta);
  const R wn_r = A::in(sc.wnow_rth), wnew_r = A::in(sc.wnew_rth);
  const R wn_v = A::in(sc.wnow_vel), wnew_v = A::in(sc.wnew_vel), cvd_o_rd = A::in(sc.cvd_o_rd);
  const float wn_vf = to_float(to_df(sc.wnow_vel)), wnew_vf = to_float(to_df(sc.wnew_vel));

  // carried values: half level k (interface above full level k), full level k-1,
  // and full level k itself (converted and time-averaged when it was level k+1)
  R ric_k = zero, tic_k = zero, tpic_k = zero, rt_k = zero;
  R zb_km1 = zero, al_km1 = zero, ps_km1 = zero, pr_km1 = zero, cp_km1 = zero, rp_km1 = zero;
  R rho_c = zero, th_c = zero, ra_c = zero, ta_c = zero, tpa_c = zero, wk_c = zero;
  // products of half level k carried from level k-1: rho_ic w, (rho theta)_ic w, beta (rho theta)_ic
  R fr_c = zero, fg_c = zero, al_c = zero;

  for (int k0 = 0; k0 < nlev; k0 += KC) {
    const int nkc = min(KC, nlev - k0);       // levels solved in this chunk
    const int nkf = min(KC + 1, nlev - k0);   // full levels with one lookahead (rho, theta)
    const int nkh = min(KC + 1, nlevp - k0);  // half levels with one lookahead (w); exner and
                                              // the tendencies are read at the chunk's levels only
    __syncthreads();
    tile_rows<KC>(T_w, a.w, nlevp, rows_c, k0, nkh);
    tile_rows<KC>(T_rho, a.rho, nlev, rows_c, k0, nkf);
    tile_rows<KC>(T_pi, a.exner, nlev, rows_c, k0, nkc);
    tile_rows<KC>(T_th, a.theta, nlev, rows_c, k0, nkf);
    tile_rows<KC>(T_dw0, a.ddt_w0, nlevp, rows_c, k0, nkc);
    tile_rows<KC>(T_dm, a.div_m, nlev, rows_c, k0, nkc);
    tile_rows<KC>(T_dt, a.div_t, nlev, rows_c, k0, nkc);
    if (corrector) {
      tile_rows<KC>(T_dw1, a.ddt_w1, nlevp, rows_c, k0, nkc);
      tile_rows<KC>(T_rp, a.rho_p, nlev, rows_c, k0, nkf);
      tile_rows<KC>(T_tp, a.theta_p, nlev, rows_c, k0, nkf);
      if (!kOwnZb) tile_levels(T_zb, kLD, a.zbl, nc, c0, k0, nkc);
    }
    if constexpr (kStage) {
      for (int i = t; i < 16 * nkf; i += kCW) cp8(L_s + i, lev_src + 16 * (size_t)k0 + i);
    }
    cp_wait();
    __syncthreads();
    if (!active) continue;
#pragma unroll 1
    for (int kk = 0; kk < nkc; ++kk) {
      const int k = k0 + kk;
      const int o = kk * kLD + t;
      if (k == 0) {
        rho_c = A::in(T_rho[o]);
        th_c = A::in(T_th[o]);
        ra_c = corrector ? add_pos(wn_r * rho_c, wnew_r * stored_in<T, R>(T_rp + o)) : rho_c;
        ta_c = corrector ? add_pos(wn_r * th_c, wnew_r * stored_in<T, R>(T_tp + o)) : th_c;
        tpa_c = ta_c - levs<R, LTH, kStage>(v, L_s, 0, k0);
        wk_c = A::in(T_w[o]);
        fr_c = ric_k * wk_c;
        fg_c = rt_k * wk_c;
        al_c = beta * rt_k;
      }
      const R rho_n = rho_c, th_n = th_c, pi_n = A::in(T_pi[o]);
      const R pr_k = pi_n - levs<R, LEX, kStage>(v, L_s, k, k0);
      // interface k+1 from full levels k and k+1 (time-averaged in the corrector)
      R ric_k1 = zero, tic_k1 = zero, tpic_k1 = zero;
      R rho_x = zero, th_x = zero, ra_x = zero, ta_x = zero, tpa_x = zero;
      if (k + 1 < nlev) {
        rho_x = A::in(T_rho[o + kLD]);
        th_x = A::in(T_th[o + kLD]);
        ra_x = corrector ? add_pos(wn_r * rho_x, wnew_r * stored_in<T, R>(T_rp + o + kLD)) : rho_x;
        ta_x = corrector ? add_pos(wn_r * th_x, wnew_r * stored_in<T, R>(T_tp + o + kLD)) : th_x;
        tpa_x = ta_x - levs<R, LTH, kStage>(v, L_s, k + 1, k0);
        const R g1 = levs<R, WG, kStage>(v, L_s, k + 1, k0), g2 = levs<R, WG2, kStage>(v, L_s, k + 1, k0);
        ric_k1 = add_pos(g1 * ra_c, g2 * ra_x);
        tic_k1 = add_pos(g1 * ta_c, g2 * ta_x);
        tpic_k1 = g1 * tpa_c + g2 * tpa_x;
      }
      const size_t ik = (size_t)k * nc + c;
      R zb;
      if (!corrector || kOwnZb) {
        zb = levs<R, CZB, kStage>(v, L_s, k, k0) * pi_n * A::inv(rho_n * th_n);
        put(a.zbl + ik, zb);
        put(eb_s + ik, pi_n - cvd_o_rd * pr_k);
      } else {
        zb = get<R>(T_zb + o);
      }
      const R wk = wk_c, wk1 = A::in(T_w[o + kLD]);
      const R rt_k1 = ric_k1 * tic_k1;
      const R fr_k1 = ric_k1 * wk1, fg_k1 = rt_k1 * wk1;
      const R rstar = rho_n - dt * stored_in<T, R>(T_dm + o) - levs<R, CR, kStage>(v, L_s, k, k0) * (fr_c - fr_k1);
      const R pstar = pr_k - zb * (levs<R, LDZ, kStage>(v, L_s, k, k0) * stored_in<T, R>(T_dt + o) + ombeta * (fg_c - fg_k1));
      const R al_k = al_c, al_k1 = beta * rt_k1;
      put(rs_s + ik, rstar);
      put(ps_s + ik, pstar);
      put(ri_s + ik, ric_k);
      put(al_s + ik, al_k);
      if (k >= 1) {
        R ddtw;
        if constexpr (std::is_same<T, float>::value) {  // FP32 tendencies: their time average in FP32
          ddtw = A::in(corrector ? fmaf(wn_vf, T_dw0[o], wnew_vf * T_dw1[o]) : T_dw0[o]);
        } else {
          ddtw = corrector ? wn_v * A::in(T_dw0[o]) + wnew_v * A::in(T_dw1[o]) : A::in(T_dw0[o]);
        }
        const R wstar = wk + dt * ddtw - (levs<R, CWX, kStage>(v, L_s, k, k0) * tic_k * (pr_km1 - pr_k) + levs<R, CB, kStage>(v, L_s, k, k0) * tpic_k);
        const R gam = levs<R, CGAM, kStage>(v, L_s, k, k0) * tic_k;
        const R am = -(gam * zb_km1 * al_km1);
        const R bm = add_pos(one, gam * al_k * add_pos(zb_km1, zb));
        const R cm = -(gam * zb * al_k1);
        const R rm = wstar - gam * (ps_km1 - pstar);
        R cpk, rpk;
        if (k == 1) {
          const R inv = A::inv(bm);
          cpk = cm * inv;
          rpk = rm * inv;
        } else {
          const R inv = A::inv(bm - am * cp_km1);
          cpk = cm * inv;
          rpk = (rm - am * rp_km1) * inv;
        }
        put(cp_s + ik, cpk);
        put(rp_s + ik, rpk);
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
      fr_c = fr_k1;
      fg_c = fg_k1;
      al_c = al_k1;
      rho_c = rho_x;
      th_c = th_x;
      wk_c = wk1;
      ra_c = ra_x;
      ta_c = ta_x;
      tpa_c = tpa_x;
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
  double* O_rho = O_w + kOut;
  double* O_pi = O_w + 2 * kOut;
  double* O_th = O_w + 3 * kOut;
  // the level-major scratch written above by this thread is read back by
  // other threads of the CTA through the asynchronous copies below
  __threadfence_block();
  // w_und of level k+1 and the fluxes rho_ic w', beta (rho theta)_ic w' at its half level
  R w_und_k1 = zero, fr_k1 = zero * zero, fa_k1 = zero * zero;
  const unsigned long long pol_last = policy_evict_first();
  for (int kend = nlev; kend > 0; kend -= KC) {
    const int k0 = max(0, kend - KC), nk = kend - k0;
    __syncthreads();
    tile_levels_last(B_cp, kCW, cp_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_rp, kCW, rp_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_rs, kCW, rs_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_ps, kCW, ps_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_ri, kCW, ri_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_al, kCW, al_s, nc, c0, k0, nk, pol_last);
    tile_levels_last(B_eb, kCW, eb_s, nc, c0, k0, nk, pol_last);
    tile_levels(B_zb, kCW, a.zbl, nc, c0, k0, nk);
    if constexpr (kStage) {
      for (int i = t; i < 16 * nk; i += kCW) cp8(L_s + i, lev_src + 16 * (size_t)k0 + i);
    }
    cp_wait();
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int kk = nk - 1; kk >= 0; --kk) {
        const int k = k0 + kk;
        const int b = kk * kCW + t;
        R w_und = zero, wd = zero;
        if (k >= 1) {
          w_und = get<R>(B_rp + b) - get<R>(B_cp + b) * w_und_k1;
          wd = w_und * levs<R, LRAY, kStage>(v, L_s, k, k0);
        }
        const R ric = get<R>(B_ri + b), al = get<R>(B_al + b), zb = get<R>(B_zb + b);
        const R fr = ric * wd, fa = al * wd;
        const R rnew = get<R>(B_rs + b) - levs<R, CRN, kStage>(v, L_s, k, k0) * (fr - fr_k1);
        const R prnew = get<R>(B_ps + b) - zb * (fa - fa_k1);
        const R thnew = levs<R, CZB, kStage>(v, L_s, k, k0) * (get<R>(B_eb + b) + cvd_o_rd * prnew) * A::inv(zb * rnew);
        const int o = kk * kLD + t;
        if (a.w_o) O_w[o] = A::out(wd);
        if (kPairs && !corrector) {
          // the mixed predictor's rho and theta_v stay double-word pairs (read by the corrector)
          *reinterpret_cast<R*>(O_rho + o) = rnew;
          *reinterpret_cast<R*>(O_th + o) = thnew;
        } else {
          O_rho[o] = A::out(rnew);
          O_th[o] = A::out(thnew);
        }
        if (a.exner_o) O_pi[o] = A::out(levs<R, LEX, kStage>(v, L_s, k, k0) + prnew);
        if constexpr (kDW) {
          // FP32 mirrors straight from the double-word values, into this
          // thread's consumed scratch slots: (w, rho - rho_ref) and theta_v - theta_ref
          float* m0 = reinterpret_cast<float*>(B_cp + b);
          m0[0] = to_float(wd);
          m0[1] = to_float(rnew - levs<R, LRHO, kStage>(v, L_s, k, k0));
          reinterpret_cast<float*>(B_rp + b)[0] = to_float(thnew - levs<R, LTH, kStage>(v, L_s, k, k0));
        }
        w_und_k1 = w_und;
        fr_k1 = fr;
        fa_k1 = fa;
      }
    }
    __syncthreads();
    if (a.w_o) store_tile<KC>(O_w, a.w_o, nlevp, c0, nc, k0, nk);
    store_tile<KC>(O_rho, a.rho_o, nlev, c0, nc, k0, nk);
    if (a.exner_o) store_tile<KC>(O_pi, a.exner_o, nlev, c0, nc, k0, nk);
    store_tile<KC>(O_th, a.theta_o, nlev, c0, nc, k0, nk);
    if constexpr (kDW) {
      if (a.m_w) mirror_chunk<KC>(B_cp, B_rp, a.m_w, a.m_rho, a.m_th, nlev, c0, nc, k0, nk);
    }
  }
  if (active) {
    if (a.w_o) a.w_o[(size_t)c * nlevp + nlev] = 0.0;
    if (a.m_w) a.m_w[(size_t)c * nlevp + nlev] = 0.0f;
  }
}

}  // namespace

// Mixed precision (FP32 stencil inputs) solves in double-word FP32 arithmetic;
// the FP64 mode in FP64.
template <class T>
using ColArith = typename std::conditional<std::is_same<T, float>::value, dws, double>::type;

cudaError_t init_column_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kernel, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set(sn_column_tiled<double, false, 8, double, 0>, smem_bytes<double, 8, false>());
  set(sn_column_tiled<double, false, 8, double, 1>, smem_bytes<double, 8, true>());
  set(sn_column_tiled<float, false, 8, dws, 0>, smem_bytes<float, 8, false>());
  set(sn_column_tiled<float, false, 8, dws, 1>, smem_bytes<float, 8, true>());
  set(sn_column_tiled<double, false, 6, double, 0>, smem_bytes<double, 6, false>());
  set(sn_column_tiled<double, false, 6, double, 1>, smem_bytes<double, 6, true>());
  set(sn_column_tiled<float, false, 6, dws, 0>, smem_bytes<float, 6, false>());
  set(sn_column_tiled<float, false, 6, dws, 1>, smem_bytes<float, 6, true>());
  set(sn_column_tiled<double, false, 4, double, 0>, smem_bytes<double, 4, false>());
  set(sn_column_tiled<double, false, 4, double, 1>, smem_bytes<double, 4, true>());
  set(sn_column_tiled<float, false, 4, dws, 0>, smem_bytes<float, 4, false>());
  set(sn_column_tiled<float, false, 4, dws, 1>, smem_bytes<float, 4, true>());
  return e;
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
    a.w_o = mixed ? nullptr : wk.w_p;  // mixed: the predicted w is read only as its FP32 mirror
    a.rho_o = wk.rho_p;
    a.exner_o = nullptr;  // the predicted exner has no reader
    a.theta_o = wk.theta_p;
    if (mixed) a.m_w = en.m.w_p;
  }
  const unsigned blocks = (unsigned)((en.g64.nc + kCW - 1) / kCW);
  const char* name = mixed ? (corrector ? "sn_column_corr_mx" : "sn_column_pred_mx")
                           : (corrector ? "sn_column_corr" : "sn_column_pred");
  using RA = ColArith<T>;
  const size_t sm4c = smem_bytes<T, 4, true>(), sm4p = smem_bytes<T, 4, false>();
  const size_t sm8c = smem_bytes<T, 8, true>(), sm8p = smem_bytes<T, 8, false>();
  const size_t sm6c = smem_bytes<T, 6, true>(), sm6p = smem_bytes<T, 6, false>();
  if (en.col_kc == 6 && corrector)
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm6c, s, (sn_column_tiled<T, false, 6, RA, 1>), en.g64.nc, en.v, en.sc, 1, a);
  else if (en.col_kc == 6)
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm6p, s, (sn_column_tiled<T, false, 6, RA, 0>), en.g64.nc, en.v, en.sc, 0, a);
  else if (en.col_kc == 4 && corrector)
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm4c, s, (sn_column_tiled<T, false, 4, RA, 1>), en.g64.nc, en.v,
                     en.sc, 1, a);
  else if (en.col_kc == 4)
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm4p, s, (sn_column_tiled<T, false, 4, RA, 0>), en.g64.nc, en.v,
                     en.sc, 0, a);
  else if (corrector)
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm8c, s, (sn_column_tiled<T, false, 8, RA, 1>), en.g64.nc, en.v,
                     en.sc, 1, a);
  else
    ICON_LAUNCH_SMEM(name, blocks, kCW, sm8p, s, (sn_column_tiled<T, false, 8, RA, 0>), en.g64.nc, en.v,
                     en.sc, 0, a);
}

template void launch_column<double>(const Engine&, int, const StateView&, const double*, const double*, cudaStream_t);
template void launch_column<float>(const Engine&, int, const StateView&, const float*, const float*, cudaStream_t);

}  // namespace icon

// ===========================================================================
// Allocation-free column solve (no counterpart in the paper).
//
// Who needs it: callers that cannot allocate device memory at the time they
// call.  A host model typically reserves nearly all device memory for its own
// arrays at start-up and leaves too little for a dycore's work arrays
// (icon_dycore_create allocates those of a whole step); it can still run the
// vertically implicit solve on arrays it owns.  The column solve needs scratch
// (the Thomas elimination planes and the vertical metrics); here it lives in
// one file-scope static device array that every GPU loading this library
// holds until the process exits.  The vertical metrics are computed on the
// device from the half-level heights and scalars passed by value as kernel
// parameters, so the call's stream work reads no host memory.
// ===========================================================================
namespace icon {
namespace {

constexpr int kNoallocMaxLev = 256;
constexpr size_t kNoallocStride = 512;                 // doubles per vertical-metric slot
constexpr size_t kNoallocCoef = 10752;                 // doubles of the vertical-metric section
constexpr size_t kNoallocLevHL = 6400;                 // offset of the double-word level table
constexpr size_t kNoallocDoubles = (size_t)8 << 20;    // 64 MiB in total
constexpr size_t kNoallocPlanes = 8;                   // 7 Thomas planes + zb
constexpr size_t kNoallocMaxPoints = (kNoallocDoubles - kNoallocCoef) / kNoallocPlanes;
static_assert(kNoallocMaxPoints == 1047232, "the limit stated in icon_dycore.h");
static_assert(8 * kNoallocStride + 8 * (kNoallocMaxLev + 1) <= kNoallocLevHL, "column coefficients fit");
static_assert(kNoallocLevHL + 16 * (kNoallocMaxLev + 1) <= kNoallocCoef, "level table fits");

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Everything the vertical metrics are derived from, passed by value (about
// 2.1 KB of kernel parameters).
struct NoallocSetup {
  int nlev;
  double dt_s, beta, rd_o_cvd, cpd, grav, ref_T0, rayleigh_coeff, damp_height;
  double z_ifc[kNoallocMaxLev + 1];
};

// double -> (hi, lo) FP32 pair, as split_hl on the host
__device__ __forceinline__ void split_pair(double x, float* out) {
  const float hi = __double2float_rn(x);
  out[0] = hi;
  out[1] = __double2float_rn(x - (double)hi);
}

// The vertical metrics, reference state, Rayleigh factors, column
// coefficients and double-word level table of icon_dycore_create, written
// into the metric section of the static array (every slot the column kernel
// reads, zeros included, so nothing is left from an earlier call).  One
// thread: about nlev sequential levels of scalar work.
__global__ void noalloc_metrics(NoallocSetup q, double* base) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int nlev = q.nlev;
  double* dz = base;
  double* inv_dz = base + kNoallocStride;
  double* inv_dzh = base + 2 * kNoallocStride;
  double* wgt = base + 3 * kNoallocStride;
  double* th_ref = base + 4 * kNoallocStride;
  double* ex_ref = base + 5 * kNoallocStride;
  double* dref = base + 6 * kNoallocStride;
  double* ray = base + 7 * kNoallocStride;
  double* colc = base + 8 * kNoallocStride;
  float* lev = reinterpret_cast<float*>(base + kNoallocLevHL);
  const double* z = q.z_ifc;
  const double H = q.cpd * q.ref_T0 / q.grav;
  for (int k = 0; k < nlev; ++k) {
    const double zm = 0.5 * (z[k] + z[k + 1]);
    dz[k] = z[k] - z[k + 1];
    inv_dz[k] = 1.0 / dz[k];
    th_ref[k] = q.ref_T0 * exp(zm / H);
  }
  for (int k = 0; k <= nlev; ++k) {
    inv_dzh[k] = 0.0;
    wgt[k] = 0.0;
    dref[k] = 0.0;
  }
  for (int k = 1; k < nlev; ++k) {
    const double zu = 0.5 * (z[k - 1] + z[k]), zl = 0.5 * (z[k] + z[k + 1]);
    inv_dzh[k] = 1.0 / (zu - zl);
    wgt[k] = (z[k] - zl) / (zu - zl);
  }
  ex_ref[nlev - 1] = exp(-0.5 * (z[nlev - 1] + z[nlev]) / H);
  for (int k = nlev - 1; k >= 1; --k) {
    const double zu = 0.5 * (z[k - 1] + z[k]), zl = 0.5 * (z[k] + z[k + 1]);
    const double th_ic = wgt[k] * th_ref[k - 1] + (1.0 - wgt[k]) * th_ref[k];
    ex_ref[k - 1] = ex_ref[k] - q.grav * (zu - zl) / (q.cpd * th_ic);
  }
  for (int k = 1; k < nlev; ++k) dref[k] = (ex_ref[k - 1] - ex_ref[k]) * inv_dzh[k];
  for (int k = 0; k <= nlev; ++k) {
    ray[k] = 1.0;
    if (q.rayleigh_coeff > 0.0 && z[k] > q.damp_height) {
      const double sn = sin(0.5 * 3.141592653589793 * (z[k] - q.damp_height) / (z[0] - q.damp_height));
      ray[k] = 1.0 / (1.0 + q.dt_s * q.rayleigh_coeff * sn * sn);
    }
  }
  for (int k = 0; k <= nlev; ++k) {
    double* cf = colc + 8 * (size_t)k;
    for (int j = 0; j < 8; ++j) cf[j] = 0.0;
    if (k < nlev) {
      cf[0] = q.dt_s * q.rd_o_cvd / dz[k];
      cf[1] = q.dt_s * (1.0 - q.beta) / dz[k];
      cf[2] = q.dt_s * q.beta / dz[k];
    }
    if (k >= 1 && k < nlev) {
      cf[3] = q.dt_s * q.cpd * (1.0 - q.beta) * inv_dzh[k];
      cf[4] = q.dt_s * q.cpd * dref[k];
      cf[5] = q.dt_s * q.cpd * q.beta * inv_dzh[k];
      cf[6] = wgt[k];
      cf[7] = 1.0 - wgt[k];
    }
    // the double-word table: colc, then exner_ref, theta_ref, dz, ray_fac
    // (no rho offset: this entry point's inputs are FP64)
    float* r = lev + 32 * (size_t)k;
    for (int j = 0; j < 32; ++j) r[j] = 0.0f;
    for (int j = 0; j < 8; ++j) split_pair(cf[j], r + 2 * j);
    if (k < nlev) {
      split_pair(ex_ref[k], r + 16);
      split_pair(th_ref[k], r + 18);
      split_pair(dz[k], r + 20);
    }
    split_pair(ray[k], r + 22);
  }
}

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Once per device, with that device current: the device address of the
// static array (its host-side name is only a stand-in) and the kernel's
// shared-memory attribute.
int noalloc_setup(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(ICON_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoallocMaxDevices)
    return report_error(ICON_ERR_CUDA, "icon_column_solve_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return report_error(ICON_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaFuncSetAttribute(sn_column_tiled<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(sn_column_tiled<double, true, kKC, dws>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSmem);
    if (e != cudaSuccess)
      return report_error(ICON_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return ICON_OK;
}

}  // namespace
}  // namespace icon

extern "C" int icon_column_solve_noalloc(int32_t n_cols, int32_t nlev, const double* z_ifc,
                                         const icon_dycore_params_t* p, const double* w, const double* rho,
                                         const double* exner, const double* theta_v, const double* rho_pred,
                                         const double* theta_pred, const double* ddt_w0, const double* ddt_w1,
                                         const double* div_m, const double* div_t, double* w_new, double* rho_new,
                                         double* exner_new, double* theta_new) {
  using namespace icon;
  const char* fn = "icon_column_solve_noalloc: ";
  if (!z_ifc || !p || !w || !rho || !exner || !theta_v || !ddt_w0 || !div_m || !div_t || !w_new || !rho_new ||
      !exner_new || !theta_new)
    return report_error(ICON_ERR_ARG, std::string(fn) + "NULL argument");
  const bool corr = rho_pred != nullptr;
  if (corr && (!theta_pred || !ddt_w1))
    return report_error(ICON_ERR_ARG, std::string(fn) + "the corrector form needs rho_pred, theta_pred and ddt_w1");
  if (n_cols < 1 || nlev < 2 || nlev > kNoallocMaxLev)
    return report_error(ICON_ERR_ARG, std::string(fn) + "need n_cols >= 1 and 2 <= nlev <= 256");
  const size_t points = (size_t)n_cols * (size_t)(nlev + 1);
  if (points > kNoallocMaxPoints)
    return report_error(ICON_ERR_ARG, std::string(fn) + "n_cols*(nlev+1) = " + std::to_string(points) +
                                          " exceeds the static scratch of " + std::to_string(kNoallocMaxPoints) +
                                          " column-levels (64 MiB)");
  for (int k = 0; k <= nlev; ++k)
    if (!std::isfinite(z_ifc[k])) return report_error(ICON_ERR_ARG, std::string(fn) + "z_ifc not finite");
  for (int k = 0; k < nlev; ++k)
    if (!(z_ifc[k] > z_ifc[k + 1])) return report_error(ICON_ERR_ARG, std::string(fn) + "z_ifc must decrease");
  if (z_ifc[nlev] != 0.0) return report_error(ICON_ERR_ARG, std::string(fn) + "z_ifc[nlev] must be 0");
  if (!(p->dtime > 0.0) || p->ndyn_substeps < 1)
    return report_error(ICON_ERR_ARG, std::string(fn) + "dtime must be > 0 and ndyn_substeps >= 1");
  if (p->precision != ICON_PREC_FP64 && p->precision != ICON_PREC_MIXED)
    return report_error(ICON_ERR_ARG, std::string(fn) + "precision must be ICON_PREC_FP64 or ICON_PREC_MIXED");

  // scalars with the same definitions as icon_dycore_create
  Scalars s{};
  s.dtime = p->dtime;
  s.dt_s = p->dtime / p->ndyn_substeps;
  s.grav = p->grav;
  s.rd = p->rd;
  s.cpd = p->cpd;
  s.cvd = p->cpd - p->rd;
  s.p00 = p->p00;
  s.beta = p->vwind_impl_wgt;
  s.wnow_vel = p->wgt_nnow_vel;
  s.wnew_vel = p->wgt_nnew_vel;
  s.wnow_rth = p->wgt_nnow_rth;
  s.wnew_rth = p->wgt_nnew_rth;
  s.exfac = p->exner_exfac;
  s.divdamp = p->divdamp_fac;
  s.rd_o_cvd = p->rd / s.cvd;
  s.cvd_o_rd = s.cvd / p->rd;
  s.hdiff_temp = p->hdiff_temp ? 1 : 0;
  NoallocSetup q{};
  q.nlev = nlev;
  q.dt_s = s.dt_s;
  q.beta = s.beta;
  q.rd_o_cvd = s.rd_o_cvd;
  q.cpd = p->cpd;
  q.grav = p->grav;
  q.ref_T0 = p->ref_T0;
  q.rayleigh_coeff = p->rayleigh_coeff;
  q.damp_height = p->damp_height;
  for (int k = 0; k <= nlev; ++k) q.z_ifc[k] = z_ifc[k];

  double* base = nullptr;
  int rc = noalloc_setup(&base);
  if (rc != ICON_OK) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(p->stream);
  // the metrics into the static array, on the device, from the by-value block
  noalloc_metrics<<<1, 32, 0, stream>>>(q, base);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(e));
  DevVert v{};
  v.nlev = nlev;
  v.dz = base;
  v.inv_dz = base + kNoallocStride;
  v.inv_dzh = base + 2 * kNoallocStride;
  v.wgt = base + 3 * kNoallocStride;
  v.theta_ref = base + 4 * kNoallocStride;
  v.exner_ref = base + 5 * kNoallocStride;
  v.dexner_ref_ic = base + 6 * kNoallocStride;
  v.ray_fac = base + 7 * kNoallocStride;
  v.colc = base + 8 * kNoallocStride;
  v.lev_hl = reinterpret_cast<const float*>(base + kNoallocLevHL);
  // every scratch plane the kernel reads is written earlier in the same call,
  // so nothing has to be cleared between calls
  ColArgs<double> a{};
  a.w = w;
  a.rho = rho;
  a.exner = exner;
  a.theta = theta_v;
  a.ddt_w0 = ddt_w0;
  a.ddt_w1 = ddt_w1;
  a.rho_p = rho_pred;
  a.theta_p = theta_pred;
  a.div_m = div_m;
  a.div_t = div_t;
  a.col = base + kNoallocCoef;
  a.zbl = a.col + 7 * points;
  a.w_o = w_new;
  a.rho_o = rho_new;
  a.exner_o = exner_new;
  a.theta_o = theta_new;
  const unsigned blocks = (unsigned)((n_cols + kCW - 1) / kCW);
  if (p->precision == ICON_PREC_MIXED)  // the mixed mode's double-word FP32 arithmetic
    sn_column_tiled<double, true, kKC, dws><<<blocks, kCW, kSmem, stream>>>(n_cols, v, s, corr ? 1 : 0, a);
  else
    sn_column_tiled<double, true><<<blocks, kCW, kSmem, stream>>>(n_cols, v, s, corr ? 1 : 0, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(e));
  if (p->synchronous) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return report_error(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(e));
  }
  return ICON_OK;
}
