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
// back-substitution.  Arranged for few FP64 operations (the FP64 pipe bounds
// this kernel): with gam_k = dt cpd beta theta_ic/dzh_k, the explicit pressure
// term is gam_k ((1-beta)/beta)(pr_k-1 - pr_k), carried in
// S_k = pr*_k + ((1-beta)/beta) pr_k together with the implicit one; the
// matrix entries use p_k = zb_k A_k and q_k = zb_k A_k+1 (A = beta (rho
// theta)_ic at the half levels); theta_ic is the reference theta at the half
// level plus the interpolated perturbation.  theta'_v from the linearised
// equation of state
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
//
// This header holds the kernel template and its helpers; kernels_column.cu
// instantiates the flat-ground forms (and the allocation-free entry point),
// kernels_column_terrain.cu the terrain-following ones.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
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
// (KC + 1) x kLD (+ over terrain the contravariant correction's tile of type
// T).  Backward (reusing it): 8 level-major scratch chunks [KC][kCW] and 4
// output tiles [KC][kLD] (+ over terrain one [KC][kLD] tile of type T).  Then
// the per-level table of a chunk: 16 slots per level, KC + 1 levels.
// kCorrTiles: room for the corrector's tiles.
template <class T, int KC, bool kCorrTiles, bool kTerr = false>
__host__ __device__ constexpr int fwd_bytes() {
  return (6 + (kCorrTiles ? 3 : 0)) * tile_doubles<KC>() * 8 +
         ((kCorrTiles ? 2 : 1) + (kTerr ? 1 : 0)) * tile_doubles<KC>() * (int)sizeof(T);
}
template <class T, int KC, bool kTerr = false>
__host__ __device__ constexpr int back_bytes() {
  return (8 * KC * kCW + 4 * KC * kLD) * 8 + (kTerr ? KC * kLD * (int)sizeof(T) : 0);
}
template <class T, int KC, bool kCorrTiles, bool kTerr = false>
__host__ __device__ constexpr int lev_offset_bytes() {
  return ((fwd_bytes<T, KC, kCorrTiles, kTerr>() > back_bytes<T, KC, kTerr>() ? fwd_bytes<T, KC, kCorrTiles, kTerr>()
                                                                               : back_bytes<T, KC, kTerr>()) +
          15) /
         16 * 16;
}
template <class T, int KC, bool kCorrTiles, bool kTerr = false>
constexpr size_t smem_bytes() {
  return (size_t)lev_offset_bytes<T, KC, kCorrTiles, kTerr>() + 16 * (size_t)(KC + 1) * sizeof(double);
}
constexpr size_t kSmem = smem_bytes<double, kKC, true>();
// CTAs of a form that fit one SM by shared memory (233 472 bytes an SM, 1 KB
// of it reserved per CTA), at most 8: the launch bound's minimum, so that the
// compiler may use the registers the shared-memory limit leaves free
template <class T, int KC, bool kCorrTiles, bool kTerr = false>
constexpr int col_min_blocks() {
  return (int)(233472 / (smem_bytes<T, KC, kCorrTiles, kTerr>() + 1024)) < 1   ? 1
         : (int)(233472 / (smem_bytes<T, KC, kCorrTiles, kTerr>() + 1024)) > 8 ? 8
                                                                              : (int)(233472 / (smem_bytes<T, KC, kCorrTiles, kTerr>() + 1024));
}

// column coefficients: CTHI the reference theta_v at the half level (theta_ic
// is it plus the interpolated perturbation); the explicit part
// of the vertical pressure-gradient term is CGAM (1 - beta)/beta.
enum { CZB = 0, CR = 1, CRN = 2, CTHI = 3, CB = 4, CGAM = 5, WG = 6, WG2 = 7 };

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
  // terrain: contravariant correction of the winds (cells, half levels)
  const T* wcc;
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

// Per-level quantity J of level k: over terrain (kTerr) this column's own
// value from the slot-major, level-major table v.colt, else levs.
template <class R, int J, bool kStaged, bool kTerr>
__device__ __forceinline__ R levc(const DevVert& v, const double* Ls, int k, int k0, int c, int nc) {
  if constexpr (kTerr) {
    return *reinterpret_cast<const R*>(v.colt + ((size_t)J * (v.nlev + 1) + k) * nc + c);
  } else {
    return levs<R, J, kStaged>(v, Ls, k, k0);
  }
}

// FP32 mirror value of a solve result: the double-word pair's leading sum,
// or the FP64 value narrowed without the FP64 pipe
__device__ __forceinline__ float mirror_f32(dws x) { return to_float(x); }
__device__ __forceinline__ float mirror_f32(double x) { return to_float(to_df(x)); }

// x - q for the terrain's contravariant correction q (type T).  In FP64 a
// plain subtraction (exact where q = 0).  In double-word arithmetic x itself
// where q is exactly zero, so that the pairs the FP64 inputs are split into (a
// truncated leading word) are not renormalised over flat ground: equal
// columns then step like the flat dycore bit for bit in either arithmetic.
// (A select in the FP64 form changes how the compiler fuses the products of
// x into multiply-adds, and with it the last bit.)
template <class R, class T>
__device__ __forceinline__ R minus_corr(R x, T q) {
  if constexpr (std::is_same<R, double>::value) {
    return x - Ar<R>::in(q);
  } else {
    return q == T(0) ? x : x - Ar<R>::in(q);
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

// A horizontal flux divergence: the mixed-precision stencils (T = float)
// store it as a double-word pair in its 8-byte slot whatever the solve's
// arithmetic R (read as the pair, or widened to FP64 exactly); else FP64.
template <class T, class R>
__device__ __forceinline__ R stored_div(const double* p) {
  if constexpr (std::is_same<T, float>::value) {
    const df x = *reinterpret_cast<const df*>(p);
    if constexpr (std::is_same<R, double>::value) {
      return f2d_exact(x.hi) + f2d_exact(x.lo);
    } else {
      return to_dws(x);
    }
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
// kTerr: per-column metrics and the solve in the contravariant velocity
// w - wcc (zero at the top and the ground, where w = wcc: the kinematic
// ground condition); the fluxes rho_ic w and the Rayleigh damping act on it.
template <class T, bool kOwnZb = false, int KC = kKC, class R = double, int kCorr = -1, bool kTerr = false>
__global__ void __launch_bounds__(kCW, (col_min_blocks<T, KC, kCorr != 0, kTerr>())) sn_column_tiled(int nc, DevVert v, Scalars sc, int corrector_arg,
                                                          ColArgs<T> a) {
  const bool corrector = kCorr < 0 ? corrector_arg != 0 : kCorr == 1;
  using A = Ar<R>;
  constexpr bool kDW = !std::is_same<R, double>::value;
  // the mixed step's engine path (FP32 stencil inputs, double-word solve)
  constexpr bool kPairs = std::is_same<T, float>::value && kDW;
  // FP32 stencils read FP32 mirrors of the solve's outputs (either arithmetic)
  constexpr bool kMirror = std::is_same<T, float>::value;
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
  T* T_wc = T_dw0 + (kCT ? 2 : 1) * kTile;  // terrain: contravariant correction
  // the per-level table is staged per chunk, except in the FP64 form of the
  // allocation-free entry, which has no FP64 copy of the table
  // (over terrain only for the FP32 mirrors' offsets of the mixed modes;
  // every physical quantity is the column's own)
  constexpr bool kStage = kTerr ? (kDW || kMirror) : (kDW || !kOwnZb);
  double* L_s = sm + lev_offset_bytes<T, KC, kCT, kTerr>() / 8;
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
  const R dt_wn_v = A::in(sc.dt_s * sc.wnow_vel), dt_wnew_v = A::in(sc.dt_s * sc.wnew_vel);
  const R cvd_o_rd = A::in(sc.cvd_o_rd), ex_o_im = A::in((1.0 - sc.beta) / sc.beta);
  const float wn_vf = to_float(to_df(sc.wnow_vel)), wnew_vf = to_float(to_df(sc.wnew_vel));
  // levels k < n_ray may be Rayleigh-damped (the factor is 1 below)
  const int n_ray = v.n_ray;

  // carried values: half level k (interface above full level k), full level k-1,
  // and full level k itself (converted and time-averaged when it was level k+1)
  R ric_k = zero, tic_k = zero, tpic_k = zero, rt_k = zero;
  R p_km1 = zero, q_km1 = zero, s_km1 = zero, cp_km1 = zero, rp_km1 = zero;
  R rho_c = zero, th_c = zero, ra_c = zero, tpa_c = zero, wk_c = zero;
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
    if constexpr (kTerr) tile_rows<KC>(T_wc, a.wcc, nlevp, rows_c, k0, nkh);
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
        const R ta_c = corrector ? add_pos(wn_r * th_c, wnew_r * stored_in<T, R>(T_tp + o)) : th_c;
        tpa_c = ta_c - levc<R, LTH, kStage, kTerr>(v, L_s, 0, k0, c, nc);
        wk_c = A::in(T_w[o]);
        const R wf = kTerr ? minus_corr(wk_c, T_wc[o]) : wk_c;
        fr_c = ric_k * wf;
        fg_c = rt_k * wf;
        al_c = beta * rt_k;
      }
      const R rho_n = rho_c, th_n = th_c, pi_n = A::in(T_pi[o]);
      const R pr_k = pi_n - levc<R, LEX, kStage, kTerr>(v, L_s, k, k0, c, nc);
      // interface k+1 from full levels k and k+1 (time-averaged in the corrector)
      R ric_k1 = zero, tic_k1 = zero, tpic_k1 = zero;
      R rho_x = zero, th_x = zero, ra_x = zero, tpa_x = zero;
      if (k + 1 < nlev) {
        rho_x = A::in(T_rho[o + kLD]);
        th_x = A::in(T_th[o + kLD]);
        ra_x = corrector ? add_pos(wn_r * rho_x, wnew_r * stored_in<T, R>(T_rp + o + kLD)) : rho_x;
        const R ta_x = corrector ? add_pos(wn_r * th_x, wnew_r * stored_in<T, R>(T_tp + o + kLD)) : th_x;
        tpa_x = ta_x - levc<R, LTH, kStage, kTerr>(v, L_s, k + 1, k0, c, nc);
        const R g1 = levc<R, WG, kStage, kTerr>(v, L_s, k + 1, k0, c, nc), g2 = levc<R, WG2, kStage, kTerr>(v, L_s, k + 1, k0, c, nc);
        ric_k1 = add_pos(g1 * ra_c, g2 * ra_x);
        // the perturbation interpolated from the levels' perturbations (no
        // cancellation against the reference), the total from it
        tpic_k1 = g1 * tpa_c + g2 * tpa_x;
        tic_k1 = levc<R, CTHI, kStage, kTerr>(v, L_s, k + 1, k0, c, nc) + tpic_k1;
      }
      const size_t ik = (size_t)k * nc + c;
      R zb;
      if (!corrector || kOwnZb) {
        zb = levc<R, CZB, kStage, kTerr>(v, L_s, k, k0, c, nc) * pi_n * A::inv(rho_n * th_n);
        put(a.zbl + ik, zb);
        put(eb_s + ik, pi_n - cvd_o_rd * pr_k);
      } else {
        zb = get<R>(T_zb + o);
      }
      const R wk = wk_c, wk1 = A::in(T_w[o + kLD]);
      const R rt_k1 = ric_k1 * tic_k1;
      const R wf1 = kTerr ? minus_corr(wk1, T_wc[o + kLD]) : wk1;
      const R fr_k1 = ric_k1 * wf1, fg_k1 = rt_k1 * wf1;
      const R rstar = rho_n - dt * stored_div<T, R>(T_dm + o) - levc<R, CR, kStage, kTerr>(v, L_s, k, k0, c, nc) * (fr_c - fr_k1);
      const R pstar = pr_k - zb * (levc<R, LDZ, kStage, kTerr>(v, L_s, k, k0, c, nc) * stored_div<T, R>(T_dt + o) + ombeta * (fg_c - fg_k1));
      const R al_k = al_c, al_k1 = beta * rt_k1;
      const R p_k = zb * al_k, q_k = zb * al_k1;
      const R s_k = pstar + ex_o_im * pr_k;
      put(rs_s + ik, rstar);
      put(ps_s + ik, pstar);
      put(ri_s + ik, ric_k);
      put(al_s + ik, al_k);
      if (k >= 1) {
        // w + dt (time-averaged tendency)
        R w0;
        if constexpr (std::is_same<T, float>::value) {  // FP32 tendencies: their time average in FP32
          w0 = wk + dt * A::in(corrector ? fmaf(wn_vf, T_dw0[o], wnew_vf * T_dw1[o]) : T_dw0[o]);
        } else {
          w0 = corrector ? (wk + dt_wn_v * A::in(T_dw0[o])) + dt_wnew_v * A::in(T_dw1[o]) : wk + dt * A::in(T_dw0[o]);
        }
        const R gam = levc<R, CGAM, kStage, kTerr>(v, L_s, k, k0, c, nc) * tic_k;
        const R rhs = (kTerr ? minus_corr(w0, T_wc[o]) : w0) - levc<R, CB, kStage, kTerr>(v, L_s, k, k0, c, nc) * tpic_k;
        const R rm = rhs - gam * (s_km1 - s_k);
        // row k: -gam p_k-1 w'_k-1 + (1 + gam (q_k-1 + p_k)) w'_k - gam q_k w'_k+1 = rm
        const R gp = gam * p_km1;
        const R inv = A::inv(add_pos(one, gam * add_pos(q_km1, p_k)) + gp * cp_km1);
        const R cpk = -(gam * q_k) * inv;
        const R rpk = (rm + gp * rp_km1) * inv;
        put(cp_s + ik, cpk);
        put(rp_s + ik, rpk);
        cp_km1 = cpk;
        rp_km1 = rpk;
      }
      p_km1 = p_k;
      q_km1 = q_k;
      s_km1 = s_k;
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
  T* W_c = reinterpret_cast<T*>(O_w + 4 * kOut);  // terrain: the chunk's contravariant correction
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
    if constexpr (kTerr) tile_rows<KC>(W_c, a.wcc, nlevp, rows_c, k0, nk);
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
          wd = k < n_ray ? w_und * levc<R, LRAY, kStage, kTerr>(v, L_s, k, k0, c, nc) : w_und;
        }
        const R ric = get<R>(B_ri + b), al = get<R>(B_al + b), zb = get<R>(B_zb + b);
        const R fr = ric * wd, fa = al * wd;
        const R rnew = get<R>(B_rs + b) - levc<R, CRN, kStage, kTerr>(v, L_s, k, k0, c, nc) * (fr - fr_k1);
        const R prnew = get<R>(B_ps + b) - zb * (fa - fa_k1);
        const R thnew = levc<R, CZB, kStage, kTerr>(v, L_s, k, k0, c, nc) * (get<R>(B_eb + b) + cvd_o_rd * prnew) * A::inv(zb * rnew);
        const int o = kk * kLD + t;
        const R wt = kTerr ? minus_corr(wd, -W_c[o]) : wd;  // w = w_con + wcc
        if (a.w_o) O_w[o] = A::out(wt);
        if (kPairs && !corrector) {
          // the mixed predictor's rho and theta_v stay double-word pairs (read by the corrector)
          *reinterpret_cast<R*>(O_rho + o) = rnew;
          *reinterpret_cast<R*>(O_th + o) = thnew;
        } else {
          O_rho[o] = A::out(rnew);
          O_th[o] = A::out(thnew);
        }
        if (a.exner_o) O_pi[o] = A::out(levc<R, LEX, kStage, kTerr>(v, L_s, k, k0, c, nc) + prnew);
        if constexpr (kMirror) {
          // FP32 mirrors straight from the solve's values, into this
          // thread's consumed scratch slots: (w, rho - rho_ref) and theta_v - theta_ref
          float* m0 = reinterpret_cast<float*>(B_cp + b);
          m0[0] = mirror_f32(wt);
          m0[1] = mirror_f32(rnew - levs<R, LRHO, kStage>(v, L_s, k, k0));
          reinterpret_cast<float*>(B_rp + b)[0] = mirror_f32(thnew - levs<R, LTH, kStage>(v, L_s, k, k0));
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
    if constexpr (kMirror) {
      if (a.m_w) mirror_chunk<KC>(B_cp, B_rp, a.m_w, a.m_rho, a.m_th, nlev, c0, nc, k0, nk);
    }
  }
  if (active) {
    // the ground: w_con = 0, so w = wcc there (0 over flat ground)
    const T wg = kTerr ? a.wcc[(size_t)c * nlevp + nlev] : T(0);
    if (a.w_o) a.w_o[(size_t)c * nlevp + nlev] = (double)wg;
    if (a.m_w) a.m_w[(size_t)c * nlevp + nlev] = (float)wg;
  }
}

// Mixed precision (FP32 stencil inputs) solves in double-word FP32 arithmetic;
// the FP64 mode in FP64.
template <class T>
using ColArith = typename std::conditional<std::is_same<T, float>::value, dws, double>::type;

// Arguments of the engine's predictor (corrector = 0: the predicted state
// into the work arrays) or corrector (the new state over st) column solve.
template <class T>
ColArgs<T> col_args(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1) {
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
  constexpr bool mixed = std::is_same<T, float>::value;
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
  return a;
}


// Launch of one column-solve form: chunk depth en.col_kc (4, 6 or 8),
// predictor or corrector, compute type T of the stencil inputs, arithmetic RA,
// flat ground or terrain.
template <class T, class RA, bool kTerr>
void launch_col_form(const Engine& en, int corrector, const ColArgs<T>& a, const char* name, cudaStream_t s) {
  const int nc = en.g64.nc;
  const unsigned blocks = (unsigned)((nc + kCW - 1) / kCW);
  switch (en.col_kc * 2 + (corrector ? 1 : 0)) {
    case 6 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 6, true, kTerr>()), s,
                       (sn_column_tiled<T, false, 6, RA, 1, kTerr>), nc, en.v, en.sc, 1, a);
      break;
    case 6 * 2:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 6, false, kTerr>()), s,
                       (sn_column_tiled<T, false, 6, RA, 0, kTerr>), nc, en.v, en.sc, 0, a);
      break;
    case 4 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 4, true, kTerr>()), s,
                       (sn_column_tiled<T, false, 4, RA, 1, kTerr>), nc, en.v, en.sc, 1, a);
      break;
    case 4 * 2:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 4, false, kTerr>()), s,
                       (sn_column_tiled<T, false, 4, RA, 0, kTerr>), nc, en.v, en.sc, 0, a);
      break;
    case 8 * 2 + 1:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 8, true, kTerr>()), s,
                       (sn_column_tiled<T, false, 8, RA, 1, kTerr>), nc, en.v, en.sc, 1, a);
      break;
    default:
      ICON_LAUNCH_SMEM(name, blocks, kCW, (smem_bytes<T, 8, false, kTerr>()), s,
                       (sn_column_tiled<T, false, 8, RA, 0, kTerr>), nc, en.v, en.sc, 0, a);
      break;
  }
}

// The dynamic shared-memory limit of the six forms of one (T, RA, kTerr).
template <class T, class RA, bool kTerr>
cudaError_t init_col_forms() {
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kernel, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set(sn_column_tiled<T, false, 8, RA, 0, kTerr>, smem_bytes<T, 8, false, kTerr>());
  set(sn_column_tiled<T, false, 8, RA, 1, kTerr>, smem_bytes<T, 8, true, kTerr>());
  set(sn_column_tiled<T, false, 6, RA, 0, kTerr>, smem_bytes<T, 6, false, kTerr>());
  set(sn_column_tiled<T, false, 6, RA, 1, kTerr>, smem_bytes<T, 6, true, kTerr>());
  set(sn_column_tiled<T, false, 4, RA, 0, kTerr>, smem_bytes<T, 4, false, kTerr>());
  set(sn_column_tiled<T, false, 4, RA, 1, kTerr>, smem_bytes<T, 4, true, kTerr>());
  return e;
}

// Kernel name of a launch (the profile tables and the autotuner key on it).
inline const char* column_name(bool mixed, bool f64col, bool terrain, int corrector) {
  if (!mixed) {
    if (terrain) return corrector ? "sn_column_corr_terrain" : "sn_column_pred_terrain";
    return corrector ? "sn_column_corr" : "sn_column_pred";
  }
  if (f64col) {
    if (terrain) return corrector ? "sn_column_corr_terrain_mx64" : "sn_column_pred_terrain_mx64";
    return corrector ? "sn_column_corr_mx64" : "sn_column_pred_mx64";
  }
  if (terrain) return corrector ? "sn_column_corr_terrain_mx" : "sn_column_pred_terrain_mx";
  return corrector ? "sn_column_corr_mx" : "sn_column_pred_mx";
}

}  // namespace
}  // namespace icon
