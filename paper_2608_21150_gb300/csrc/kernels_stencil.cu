// Stencil kernels of one dycore step (rows A1-A6, A8-A10), templated on the
// compute type T: double (FP64 mode) or float (mixed mode, row A12).
//
// Layout: level-contiguous X[h * nk + k] (k = 0 at the model top); one thread
// per (horizontal point, level), flattened so that the 32 lanes of a warp
// cover consecutive levels of one or two columns (the FP32 forms of five
// gather-heavy kernels: one warp per point instead, see blocks_by_point).
// Neighbour gathers X[nbr * nk + k] are coalesced runs of consecutive levels.
//
// Mixed mode: the stencils read FP32 mirrors of the state (vn, w and the
// perturbations rho - rho_ref, theta_v - theta_ref) and compute in FP32,
// except the exner difference of the horizontal pressure gradient (double-
// word); prognostic updates stay FP64 (the FP64 state plus an FP32 increment)
// and rewrite the mirrors; flux divergences are summed in double-word FP32 so
// that every edge flux is one value shared by its two cells (mass conserved
// to about 2^-48), and stored as the pair for the column solve.  FP64<->FP32
// conversions run on the FP64 pipe on this GPU, so they are done with integer
// operations, once per value by its writer, never per gather.
#include <cuda_runtime.h>

#include <type_traits>

#include "dfloat.cuh"
#include "kernels.h"

namespace icon {

thread_local Prof* g_prof = nullptr;

namespace {

template <class T>
constexpr bool kMixed = std::is_same<T, float>::value;

// FP64 <-> FP32 without the FP64 pipe (mixed mode): exact widening, and
// narrowing through the double-word split (round to nearest up to rare
// double-rounding ties)
__device__ __forceinline__ double f2d(float x) { return f2d_exact(x); }
__device__ __forceinline__ float d2f(double x) { return to_float(to_df(x)); }

__device__ __forceinline__ bool flat_index(int n_h, int nk, int& h, int& k) {
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)n_h * (unsigned)nk) return false;
  h = (int)(i / (unsigned)nk);
  k = (int)(i - (unsigned)h * (unsigned)nk);
  return true;
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// a * b + c with one rounding, in the compute type
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// Second launch shape, used by the FP32 forms of the kernels whose per-point
// gathers dominate (va_edge_pre, va_cell_w, sn_cell_div, sn_cell_fluxdiv,
// sn_edge_corr): one warp per horizontal point, its lanes striding over the
// levels, so the point's neighbour indices and weights are loaded once per
// warp.  Not used for FP64, where 90 levels fill only 90 of 96 lane slots of
// the saturated FP64 pipe, nor for the kernels that measured slower with it.
__device__ __forceinline__ int warp_point() { return (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); }
__device__ __forceinline__ int lane_id() { return (int)(threadIdx.x & 31u); }
inline unsigned blocks_for_points(long long n_points, int threads) {
  const int warps = threads / 32;
  return (unsigned)((n_points + warps - 1) / warps);
}
// CTAs of a kernel over n_h points and nk levels in the shape of its type
template <class T>
unsigned blocks_by_point(long long n_h, int nk, int threads) {
  return kMixed<T> ? blocks_for_points(n_h, threads) : blocks_for(n_h * nk, threads);
}
// CTAs of a two-shape kernel: shape 1 one warp per point, 0 one thread per (point, level)
inline unsigned blocks_by_shape(int shape, long long n_h, int nk, int threads) {
  return shape ? blocks_for_points(n_h, threads) : blocks_for(n_h * nk, threads);
}

constexpr int kThreads = 256;

// threads per CTA of stencil kernel `id` from the autotuner's table (0: default)
inline int tuned(const int* threads, int id) { return threads && threads[id] > 0 ? threads[id] : kThreads; }
#define TH(id) tuned(threads, id)
// tile shape of a two-shape kernel from the autotuner's table (-1: the
// compute type's default, one warp per point in FP32, one thread per
// (point, level) in FP64)
template <class T>
inline int shaped(const int* shapes, int id) {
  return shapes && shapes[id] >= 0 ? shapes[id] : (kMixed<T> ? 1 : 0);
}
#define SH(id) shaped<T>(shapes, id)

template <class T>
const char* kname(const char* f64, const char* f32) {
  return kMixed<T> ? f32 : f64;
}

// -------------------------------------------------------------------------
// A1: tangential wind and edge kinetic energy
//   vt = sum_j vt_w[j] vn[e_j] (Perot reconstruction averaged over the two
//   cells, projected on t_e), K_e = (vn^2 + vt^2)/2, stored as 2 K_e (the
//   1/2 is folded into the gradient's stored factor 1/(2 d_e))
// -------------------------------------------------------------------------
// Also vn at the half levels, vn_ie (interpolated inside with the level
// weights -- the edge weights wgt_e over terrain -- the top level's value at the
// top and the lowest level's at the ground), for the edge tendency kernel.
// Both tile shapes evaluate every (edge, level) with the same explicit FMAs
// (va_edge_pre_at), so the autotuner's choice of shape does not change a bit.
template <class T>
__device__ __forceinline__ void va_edge_pre_at(const VertT<T>& v, int e, int k, int nlev, const T* x0, const T* x1,
                                               const T* x2, const T* x3, const T* x4, const T* w, T* vt, T* ekin,
                                               T* vn_ie, const T* wgt_e) {
  const int nlevp = nlev + 1;
  const T vne = x0[k];
  T t = w[0] * vne;
  t = fmat(w[1], x1[k], t);
  t = fmat(w[2], x2[k], t);
  t = fmat(w[3], x3[k], t);
  t = fmat(w[4], x4[k], t);
  vt[(size_t)e * nlev + k] = t;
  ekin[(size_t)e * nlev + k] = fmat(vne, vne, t * t);
  const T wg = wgt_e ? wgt_e[(size_t)e * nlevp + k] : v.wgt[k];
  vn_ie[(size_t)e * nlevp + k] = k == 0 ? vne : fmat(wg, x0[k - 1] - vne, vne);
  if (k == nlev - 1) vn_ie[(size_t)e * nlevp + nlev] = vne;
}

template <class T>
__global__ void va_edge_pre(GridT<T> g, VertT<T> v, const T* __restrict__ vn, T* __restrict__ vt,
                            T* __restrict__ ekin, T* __restrict__ vn_ie, const T* __restrict__ wgt_e, int shape) {
  const int nlev = v.nlev;
  if (shape) {  // one warp per edge, its lanes over the levels
    const int e = warp_point();
    if (e >= g.ne) return;
    const T* w = g.vt_w + 5 * (size_t)e;
    const T wl[5] = {w[0], w[1], w[2], w[3], w[4]};
    const int* q = g.e2c2e + 4 * (size_t)e;
    const T* x0 = vn + (size_t)e * nlev;
    const T* x1 = vn + (size_t)q[0] * nlev;
    const T* x2 = vn + (size_t)q[1] * nlev;
    const T* x3 = vn + (size_t)q[2] * nlev;
    const T* x4 = vn + (size_t)q[3] * nlev;
    for (int k = lane_id(); k < nlev; k += 32) va_edge_pre_at(v, e, k, nlev, x0, x1, x2, x3, x4, wl, vt, ekin, vn_ie, wgt_e);
    return;
  }
  int e, k;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const int* q = g.e2c2e + 4 * (size_t)e;
  va_edge_pre_at(v, e, k, nlev, vn + (size_t)e * nlev, vn + (size_t)q[0] * nlev, vn + (size_t)q[1] * nlev,
                 vn + (size_t)q[2] * nlev, vn + (size_t)q[3] * nlev, g.vt_w + 5 * (size_t)e, vt, ekin, vn_ie, wgt_e);
}

// -------------------------------------------------------------------------
// A1-A2 over terrain: contravariant correction at cell half levels, the
// vertical velocity of a parcel that follows the coordinate surface,
//   wcc = sum_e q_e (vn_ie dz/dn + vt_ie dz/dt)
// with vn, vt interpolated to the edge half levels by the edge weights (the
// lowest full level's values at the ground; vn_ie from va_edge_pre; the
// slopes vanish at the flat model top, where wcc = 0).
// -------------------------------------------------------------------------
template <class T>
__global__ void va_concorr(GridT<T> g, VertT<T> v, TerrT<T> tr, const T* __restrict__ vn_ie,
                           const T* __restrict__ vt, T* __restrict__ wcc) {
  int c, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.nc, nlevp, c, k)) return;
  T s = 0;
  if (k > 0) {
    const int* ce = g.c2e + 3 * (size_t)c;
    const T* q = g.e2c_w + 3 * (size_t)c;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int e = ce[j];
      const T* y = vt + (size_t)e * nlev;
      const size_t ih = (size_t)e * nlevp + k;
      const T a = vn_ie[ih];
      const T b = k == nlev ? y[nlev - 1] : y[k] + tr.wgt_e[ih] * (y[k - 1] - y[k]);
      s += q[j] * (a * tr.ddxn_ifc[ih] + b * tr.ddxt_ifc[ih]);
    }
  }
  wcc[(size_t)c * nlevp + k] = s;
}

// -------------------------------------------------------------------------
// A2: cells: K_c = sum q_e K_e  (and, in the corrector, the divergence-damping
//     Laplacian dd2 = lapc(div vn*));  vertices: zeta = curl vn (full levels),
//     w_v = sum r_c w_c (half levels).  One launch over nc*nlev + nv*(nlev+1).
// -------------------------------------------------------------------------
// Also, per cell and full level, wq = w_k + w_k+1 (over terrain the
// contravariant w - wcc): the edge tendency's mean of four w is then the
// sum of its two cells' wq, computed once per cell instead of once per edge.
// In FP64 the Laplacian is sum L_j dd_j - (sum L_j) dd_c: fewer FP64
// operations (the damping increment is a small part of vn, so the
// cancellation in the sum costs nothing measurable); FP32 keeps the
// differences.
template <class T>
__global__ void va_cell_vert(GridT<T> g, VertT<T> v, const T* __restrict__ vn, const T* __restrict__ w,
                             const T* __restrict__ ekin_e, T* __restrict__ ekin_c, const T* __restrict__ divd,
                             T* __restrict__ divd2, T* __restrict__ zeta, T* __restrict__ w_v, T* __restrict__ wq,
                             const T* __restrict__ wcc) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlev;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)c * nlev);
    const int* ce = g.c2e + 3 * (size_t)c;
    const T* q = g.e2c_w + 3 * (size_t)c;
    T s = q[0] * ekin_e[(size_t)ce[0] * nlev + k];
    s += q[1] * ekin_e[(size_t)ce[1] * nlev + k];
    s += q[2] * ekin_e[(size_t)ce[2] * nlev + k];
    ekin_c[i] = s;
    const T* wc = w + (size_t)c * nlevp;
    if (wcc) {
      const T* qc = wcc + (size_t)c * nlevp;
      wq[i] = (wc[k] - qc[k]) + (wc[k + 1] - qc[k + 1]);
    } else {
      wq[i] = wc[k] + wc[k + 1];
    }
    if (divd2) {
      const int* cc = g.c2e2c + 3 * (size_t)c;
      const T* L = g.lap_c + 3 * (size_t)c;
      const T dc = divd[i];
      const T d0 = divd[(size_t)cc[0] * nlev + k], d1 = divd[(size_t)cc[1] * nlev + k],
              d2 = divd[(size_t)cc[2] * nlev + k];
      if constexpr (kMixed<T>) {
        T r = L[0] * (d0 - dc);
        r += L[1] * (d1 - dc);
        r += L[2] * (d2 - dc);
        divd2[i] = r;
      } else {
        divd2[i] = fmat(L[2], d2, fmat(L[1], d1, fmat(L[0], d0, -(g.lap_s[c] * dc))));
      }
    }
    return;
  }
  i -= ncell;
  if (i >= (unsigned)g.nv * nlevp) return;
  int vx = (int)(i / (unsigned)nlevp), k = (int)(i - (unsigned)vx * nlevp);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const int* vc = g.v2c + 6 * (size_t)vx;
  const T* cw = g.curl_v + 6 * (size_t)vx;
  const T* rw = g.c2v_w + 6 * (size_t)vx;
  if (k < nlev) {
    T z = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) z += cw[j] * vn[(size_t)ve[j] * nlev + k];
    zeta[(size_t)vx * nlev + k] = z;
  }
  T s = 0;
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
// Over terrain (kTerr): edge interpolation weights and layer thicknesses, and
// the contravariant velocity w - wcc as the advecting vertical velocity.
// Arithmetic arranged for few FP64 instructions (the FP64 mode is bound by
// GB300's FP64 issue rate): wbar dvn/dz = (wq_c0 + wq_c1) (vn_ie_k -
// vn_ie_k+1) dz^-1/4 with the cells' sums of two w from va_cell_vert and
// dz^-1/4 stored, the Coriolis term's 1/2 folded into a multiply-add, the
// gradient of 2K times 1/(2 d) into the final multiply-add.  gw_e is stored
// times d_e (its 1/d_e is folded into va_cell_w's weights).
template <class T, bool kTerr = false>
__global__ void va_edge_tend(GridT<T> g, VertT<T> v, const T* __restrict__ vn_ie, const T* __restrict__ w,
                             const T* __restrict__ vt, const T* __restrict__ ekin_c, const T* __restrict__ zeta,
                             const T* __restrict__ w_v, T* __restrict__ ddt_vn, T* __restrict__ gw_e, TerrT<T> tr,
                             const T* __restrict__ wq) {
  int e, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.ne, nlevp, e, k)) return;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const T* vte = vt + (size_t)e * nlev;
  const T vnie_k = vn_ie[(size_t)e * nlevp + k];
  if (k < nlev) {
    const int vm = g.e2v[2 * e], vp = g.e2v[2 * e + 1];
    const T vnie_k1 = vn_ie[(size_t)e * nlevp + k + 1];
    const T ws = wq[(size_t)c0 * nlev + k] + wq[(size_t)c1 * nlev + k];
    const T qdz = kTerr ? tr.qdz_e[(size_t)e * nlev + k] : v.qdz[k];
    const T adv = (ws * (vnie_k - vnie_k1)) * qdz;
    const T zf = fmat(T(0.5), zeta[(size_t)vm * nlev + k] + zeta[(size_t)vp * nlev + k], g.f_e[e]);
    const T dk = ekin_c[(size_t)c0 * nlev + k] - ekin_c[(size_t)c1 * nlev + k];
    ddt_vn[(size_t)e * nlev + k] = fmat(dk, g.hinv_d[e], fmat(zf, vte[k], -adv));
  }
  T gw = 0;
  if (k > 0 && k < nlev) {
    const int vm = g.e2v[2 * e], vp = g.e2v[2 * e + 1];
    const T wg = kTerr ? tr.wgt_e[(size_t)e * nlevp + k] : v.wgt[k];
    const T vtie = vte[k] + wg * (vte[k - 1] - vte[k]);
    const T dwn = w[(size_t)c1 * nlevp + k] - w[(size_t)c0 * nlevp + k];
    const T dwt = (w_v[(size_t)vp * nlevp + k] - w_v[(size_t)vm * nlevp + k]) * g.d_o_l[e];
    gw = fmat(vnie_k, dwn, vtie * dwt);
  }
  gw_e[(size_t)e * nlevp + k] = gw;
}

// -------------------------------------------------------------------------
// A4: w advective tendency at interior half levels (0 at top and ground)
//   ddt_w = -sum q_e gw_e - w (wf_{k-1} - wf_k)/dzh,  wf full-level averages
//   (q_e/d_e stored: gw_e holds the advection times d_e)
// -------------------------------------------------------------------------
// Over terrain (kTerr): advected by w - wcc, per-cell half-level spacing.
// Both tile shapes evaluate every (cell, half level) with va_cell_w_at.
template <class T, bool kTerr>
__device__ __forceinline__ T va_cell_w_at(const VertT<T>& v, const TerrT<T>& tr, int c, int k, int nlev,
                                          const T* g0, const T* g1, const T* g2, const T* q, const T* wc,
                                          const T* wcc) {
  if (k == 0 || k >= nlev) return T(0);
  const T h = fmat(q[2], g2[k], fmat(q[1], g1[k], q[0] * g0[k]));
  // the difference of the full-level means above and below, (w_k-1 - w_k+1) / 2,
  // with the 1/2 folded into the stored 1/(2 dzh)
  T wa, qd;
  if constexpr (kTerr) {
    const size_t ih = (size_t)c * (nlev + 1) + k;
    wa = wc[k] - wcc[ih];
    qd = tr.qdzh_c[ih];
  } else {
    wa = wc[k];
    qd = v.qdzh[k];
  }
  return fmat(-(wa * (wc[k - 1] - wc[k + 1])), qd, -h);
}

template <class T, bool kTerr = false>
__global__ void va_cell_w(GridT<T> g, VertT<T> v, const T* __restrict__ w, const T* __restrict__ gw_e,
                          T* __restrict__ ddt_w, TerrT<T> tr, const T* __restrict__ wcc, int shape) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (shape) {  // one warp per cell, its lanes over the half levels
    const int c = warp_point();
    if (c >= g.nc) return;
    const int* ce = g.c2e + 3 * (size_t)c;
    const T* qp = g.e2c_wd + 3 * (size_t)c;
    const T q[3] = {qp[0], qp[1], qp[2]};
    const T* g0 = gw_e + (size_t)ce[0] * nlevp;
    const T* g1 = gw_e + (size_t)ce[1] * nlevp;
    const T* g2 = gw_e + (size_t)ce[2] * nlevp;
    const T* wc = w + (size_t)c * nlevp;
    for (int k = lane_id(); k < nlevp; k += 32)
      ddt_w[(size_t)c * nlevp + k] = va_cell_w_at<T, kTerr>(v, tr, c, k, nlev, g0, g1, g2, q, wc, wcc);
    return;
  }
  int c, k;
  if (!flat_index(g.nc, nlevp, c, k)) return;
  const int* ce = g.c2e + 3 * (size_t)c;
  ddt_w[(size_t)c * nlevp + k] =
      va_cell_w_at<T, kTerr>(v, tr, c, k, nlev, gw_e + (size_t)ce[0] * nlevp, gw_e + (size_t)ce[1] * nlevp,
                             gw_e + (size_t)ce[2] * nlevp, g.e2c_wd + 3 * (size_t)c, w + (size_t)c * nlevp, wcc);
}

// -------------------------------------------------------------------------
// A1-A4 in one launch (mixed precision, flat ground): one CTA per patch of
// consecutive cells (the refinement order makes patches compact), chunks of
// kVaL levels.  Per chunk, vn on every edge the patch reads and w on every
// cell it reads come into shared memory (coalesced runs of levels); then, one
// thread per edge, cell or vertex looping over the chunk's levels: vt and 2K
// on the edges of the patch's cells and their neighbours, 2K at those cells,
// vorticity and w at the vertices, the vn tendency and w's horizontal
// advection on the own cells' edges, the w tendency of the own cells -- each
// stage from shared memory, where the four kernels above pass through HBM.
// Results are staged in shared memory and stored as runs of levels.  Halo
// values are computed again by every patch that needs them; an edge's
// tendency and vt are written by the patch of its first cell.  Local indices
// and the grid factors come in patch order (16-bit index rows, FP32 factor
// rows), so every item's table is one or two vector loads per chunk.  Every
// value is the same expression as in the four kernels (the same bits).
// -------------------------------------------------------------------------
constexpr int kVaL = 8;          // levels per chunk
constexpr int kVaS = kVaL + 1;   // shared-memory stride of a per-item run of L or L + 1 levels (odd)
constexpr int kVaSn = kVaL + 3;  // stride of the staged vn and w runs of L + 2 levels (odd)
constexpr int kVaThreads = 512;

__host__ __device__ inline size_t va_fused_smem_floats(int max_e0, int max_e1, int max_c3, int max_c0, int max_v3,
                                                       int max_e4) {
  return 2 * (size_t)kVaSn * ((size_t)max_e0 + max_c0) +
         (size_t)kVaS * (2 * (size_t)max_e1 + 2 * (size_t)max_e4 + max_c3 + 2 * (size_t)max_v3);
}

__device__ __forceinline__ int lo16(unsigned x) { return (int)(x & 0xffffu); }
__device__ __forceinline__ int hi16(unsigned x) { return (int)(x >> 16); }

// 4-byte asynchronous global->shared copy; cp_commit closes the thread's
// group, cp_wait_all waits for every group it issued
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__global__ void __launch_bounds__(kVaThreads, 2) va_fused(GridT<float> g, VertT<float> v, VaPatchT pt,
                                                          const float* __restrict__ vn, const float* __restrict__ w,
                                                          float* __restrict__ vt_out, float* __restrict__ ddt_vn,
                                                          float* __restrict__ ddt_w, const float* __restrict__ divd,
                                                          float* __restrict__ divd2) {
  extern __shared__ float sf[];
  constexpr int L = kVaL, S = kVaS, Sn = kVaSn;
  const int p = blockIdx.x;
  const int nlev = v.nlev, nlevp = nlev + 1;
  const int e0a = pt.off_e0[p], ne0 = pt.off_e0[p + 1] - e0a;
  const int e1a = pt.off_e1[p], ne1 = pt.off_e1[p + 1] - e1a;
  const int c0a = pt.off_c0[p], nc0 = pt.off_c0[p + 1] - c0a, nc3 = pt.n_c3[p];
  const int v3a = pt.off_v3[p], nv3 = pt.off_v3[p + 1] - v3a;
  const int e4a = pt.off_e4[p], ne4 = pt.off_e4[p + 1] - e4a, nw4 = pt.n_w4[p];
  const int c_begin = p * pt.P, ncown = min(pt.P, g.nc - c_begin);
  // two stages of [e0][Sn] vn at full levels k0-1 .. k0+L and [c0][Sn] w at
  // half levels k0-1 .. k0+L: the next chunk's copies run during this one
  const size_t stage = (size_t)(pt.max_e0 + pt.max_c0) * Sn;
  float* vt_s = sf + 2 * stage;                // [e1][S]: vt at full levels k0-1 .. k0+L-1
  float* ek_s = vt_s + (size_t)pt.max_e1 * S;  // [e1][S]: 2K at full levels k0 .. k0+L-1; then ddt_vn of E4
  float* vi_s = ek_s + (size_t)pt.max_e1 * S;  // [e4][S]: vn at half levels k0 .. k0+L
  float* gw_s = vi_s + (size_t)pt.max_e4 * S;  // [e4][S]: w's horizontal advection, half levels k0 .. k0+L-1
  float* kc_s = gw_s + (size_t)pt.max_e4 * S;  // [c3][S]: 2K at the cells; then ddt_w of the own cells
  float* ze_s = kc_s + (size_t)pt.max_c3 * S;  // [v3][S]: vorticity, full levels
  float* wv_s = ze_s + (size_t)pt.max_v3 * S;  // [v3][S]: w at the vertices, half levels
  float* dv_s = ek_s;
  float* dw_s = kc_s;
  // consecutive threads copy consecutive levels of one row (coalesced)
  auto issue = [&](int kc, float* vs) {
    float* ws = vs + (size_t)pt.max_e0 * Sn;
    for (int i = threadIdx.x; i < (ne0 + nc0) * (L + 2); i += blockDim.x) {
      const int it = i / (L + 2), lv = i - it * (L + 2);
      if (it < ne0) {
        const int k = min(max(kc - 1 + lv, 0), nlev - 1);
        cp_async4(vs + it * Sn + lv, vn + (size_t)pt.e0_g[e0a + it] * nlev + k);
      } else {
        const int kh = min(max(kc - 1 + lv, 0), nlev);
        const int ic = it - ne0;
        cp_async4(ws + ic * Sn + lv, w + (size_t)pt.c0_g[c0a + ic] * nlevp + kh);
      }
    }
    cp_commit();
  };
  issue(0, sf);
  for (int k0 = 0, b = 0; k0 <= nlev + L; k0 += L, b ^= 1) {
    cp_wait_all();
    __syncthreads();
    if (k0 > 0) {  // the previous chunk's w tendencies (own cells), coalesced along the levels
      const int kp = k0 - L;
      for (int i = threadIdx.x; i < ncown * L; i += blockDim.x) {
        const int it = i / L, lv = i - it * L, k = kp + lv;
        if (k <= nlev) ddt_w[(size_t)(c_begin + it) * nlevp + k] = dw_s[it * S + lv];
      }
    }
    if (k0 > nlev) break;
    if (k0 + L <= nlev) issue(k0 + L, sf + (b ^ 1) * stage);
    const float* vn_s = sf + b * stage;
    const float* w_s = vn_s + (size_t)pt.max_e0 * Sn;
    // A1: vt and 2K on the E1 edges; vn at the half levels of the E4 edges
    for (int i = threadIdx.x; i < ne1 + ne4; i += blockDim.x) {
      if (i < ne1) {
        const int it = i;
        const uint4 nb = *reinterpret_cast<const uint4*>(pt.e1_i + 8 * (size_t)(e1a + it));
        const float* n0 = vn_s + lo16(nb.x) * Sn;
        const float* n1 = vn_s + hi16(nb.x) * Sn;
        const float* n2 = vn_s + lo16(nb.y) * Sn;
        const float* n3 = vn_s + hi16(nb.y) * Sn;
        const float* n4 = vn_s + lo16(nb.z) * Sn;
        const float* wt = pt.e1_w + 5 * (size_t)(e1a + it);
        const float w0 = wt[0], w1 = wt[1], w2 = wt[2], w3 = wt[3], w4 = wt[4];
#pragma unroll
        for (int lv = 0; lv <= L; ++lv) {
          const int k = k0 - 1 + lv;
          if (k < 0 || k >= nlev) continue;
          const float vne = n0[lv];
          float t = w0 * vne;
          t = fmat(w1, n1[lv], t);
          t = fmat(w2, n2[lv], t);
          t = fmat(w3, n3[lv], t);
          t = fmat(w4, n4[lv], t);
          vt_s[it * S + lv] = t;
          if (lv >= 1) ek_s[it * S + lv - 1] = fmat(vne, vne, t * t);
        }
      } else {
        const int it = i - ne1;
        const float* x = vn_s + (int)pt.e4_i[8 * (size_t)(e4a + it) + 1] * Sn;
#pragma unroll
        for (int lv = 0; lv <= L; ++lv) {
          const int kh = k0 + lv;
          if (kh > nlev) break;
          float vi;
          if (kh == 0) {
            vi = x[lv + 1];
          } else if (kh == nlev) {
            vi = x[lv];
          } else {
            const float vne = x[lv + 1];
            vi = fmat(v.wgt[kh], x[lv] - vne, vne);
          }
          vi_s[it * S + lv] = vi;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nw4 * L; i += blockDim.x) {  // vt of the edges this patch writes
      const int it = i / L, lv = i - it * L, k = k0 + lv;
      if (k < nlev) vt_out[(size_t)pt.e4_g[e4a + it] * nlev + k] = vt_s[(int)pt.e4_i[8 * (size_t)(e4a + it)] * S + lv + 1];
    }
    if (divd2) {  // the corrector's divergence-damping Laplacian at the own cells
      for (int i = threadIdx.x; i < ncown * L; i += blockDim.x) {
        const int it = i / L, lv = i - it * L, k = k0 + lv;
        if (k >= nlev) continue;
        const int c = c_begin + it;
        const int* cc = g.c2e2c + 3 * (size_t)c;
        const float* Lw = g.lap_c + 3 * (size_t)c;
        const size_t ic = (size_t)c * nlev + k;
        const float dc = divd[ic];
        const float d0 = divd[(size_t)cc[0] * nlev + k], d1 = divd[(size_t)cc[1] * nlev + k],
                    d2 = divd[(size_t)cc[2] * nlev + k];
        float r = Lw[0] * (d0 - dc);
        r += Lw[1] * (d1 - dc);
        r += Lw[2] * (d2 - dc);
        divd2[ic] = r;
      }
    }
    // A2: 2K at the C3 cells (all levels of the chunk); vorticity and w at the
    // V3 vertices (each vertex in two halves of the chunk's levels)
    for (int i = threadIdx.x; i < nc3 + 2 * nv3; i += blockDim.x) {
      if (i < nc3) {
        const int it = i;
        const uint2 ce = *reinterpret_cast<const uint2*>(pt.c3_i + 4 * (size_t)(c0a + it));
        const float* k0p = ek_s + lo16(ce.x) * S;
        const float* k1p = ek_s + hi16(ce.x) * S;
        const float* k2p = ek_s + lo16(ce.y) * S;
        const float4 q = *reinterpret_cast<const float4*>(pt.c3_w + 4 * (size_t)(c0a + it));
#pragma unroll
        for (int lv = 0; lv < L; ++lv) {
          const int k = k0 + lv;
          if (k >= nlev) break;
          float sk = q.x * k0p[lv];
          sk += q.y * k1p[lv];
          sk += q.z * k2p[lv];
          kc_s[it * S + lv] = sk;
        }
      } else {
        const int it = (i - nc3) >> 1, l0 = ((i - nc3) & 1) * (L / 2);
        const uint4* xi = reinterpret_cast<const uint4*>(pt.v3_i + 16 * (size_t)(v3a + it));
        const uint4 xa = xi[0], xb = xi[1];
        const float4* wp = reinterpret_cast<const float4*>(pt.v3_w + 12 * (size_t)(v3a + it));
        const float4 wa = wp[0], wb = wp[1], wc = wp[2];
        const float* ep[6] = {vn_s + lo16(xa.x) * Sn + 1, vn_s + hi16(xa.x) * Sn + 1, vn_s + lo16(xa.y) * Sn + 1,
                              vn_s + hi16(xa.y) * Sn + 1, vn_s + lo16(xa.z) * Sn + 1, vn_s + hi16(xa.z) * Sn + 1};
        const float* cp[6] = {w_s + lo16(xa.w) * Sn + 1, w_s + hi16(xa.w) * Sn + 1, w_s + lo16(xb.x) * Sn + 1,
                              w_s + hi16(xb.x) * Sn + 1, w_s + lo16(xb.y) * Sn + 1, w_s + hi16(xb.y) * Sn + 1};
        const float cwl[6] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y};
        const float rwl[6] = {wb.z, wb.w, wc.x, wc.y, wc.z, wc.w};
#pragma unroll
        for (int j = 0; j < L / 2; ++j) {
          const int lv = l0 + j, k = k0 + lv;
          if (k > nlev) break;
          if (k < nlev) {
            float z = 0;
#pragma unroll
            for (int m = 0; m < 6; ++m) z += cwl[m] * ep[m][lv];
            ze_s[it * S + lv] = z;
          }
          float sw = 0;
#pragma unroll
          for (int m = 0; m < 6; ++m) sw += rwl[m] * cp[m][lv];
          wv_s[it * S + lv] = sw;
        }
      }
    }
    __syncthreads();
    // A3: the vn tendency (edges this patch writes) and w's horizontal
    // advection (times d) on the E4 edges, each edge in two halves of the levels
    for (int i = threadIdx.x; i < 2 * ne4; i += blockDim.x) {
      const int it = i >> 1, l0 = (i & 1) * (L / 2);
      const uint4 x = *reinterpret_cast<const uint4*>(pt.e4_i + 8 * (size_t)(e4a + it));
      const float4 cf = *reinterpret_cast<const float4*>(pt.e4_w + 4 * (size_t)(e4a + it));
      const float* vt1 = vt_s + lo16(x.x) * S;
      const int lc0 = lo16(x.y), lc1 = hi16(x.y);
      const float* kc0 = kc_s + lc0 * S;
      const float* kc1 = kc_s + lc1 * S;
      const float* w0 = w_s + lc0 * Sn;
      const float* w1 = w_s + lc1 * Sn;
      const float* zm = ze_s + lo16(x.z) * S;
      const float* zp = ze_s + hi16(x.z) * S;
      const float* wvm = wv_s + lo16(x.z) * S;
      const float* wvp = wv_s + hi16(x.z) * S;
      const bool own = it < nw4;
      const float* vie = vi_s + it * S;
#pragma unroll
      for (int j = 0; j < L / 2; ++j) {
        const int lv = l0 + j, k = k0 + lv;
        if (k > nlev) break;
        const float vnie_k = vie[lv];
        if (k < nlev && own) {
          const float vnie_k1 = vie[lv + 1];
          const float ws = (w0[lv + 1] + w0[lv + 2]) + (w1[lv + 1] + w1[lv + 2]);
          const float adv = (ws * (vnie_k - vnie_k1)) * v.qdz[k];
          const float zf = fmat(0.5f, zm[lv] + zp[lv], cf.x);
          const float dk = kc0[lv] - kc1[lv];
          dv_s[it * S + lv] = fmat(dk, cf.y, fmat(zf, vt1[lv + 1], -adv));
        }
        float gw = 0;
        if (k > 0 && k < nlev) {
          const float wg = v.wgt[k];
          const float vtk = vt1[lv + 1];
          const float vtie = vtk + wg * (vt1[lv] - vtk);
          const float dwn = w1[lv + 1] - w0[lv + 1];
          const float dwt = (wvp[lv] - wvm[lv]) * cf.z;
          gw = fmat(vnie_k, dwn, vtie * dwt);
        }
        gw_s[it * S + lv] = gw;
      }
    }
    __syncthreads();
    // A4: the w tendency of the own cells, each cell in four quarters of the
    // levels (stored at the next chunk's start); the vn tendencies of the
    // edges this patch writes
    for (int i = threadIdx.x; i < 4 * ncown; i += blockDim.x) {
      const int it = i >> 2, l0 = (i & 3) * (L / 4);
      const int c = c_begin + it;
      const uint2 ce = *reinterpret_cast<const uint2*>(pt.own_i + 4 * (size_t)c);
      const float* g0 = gw_s + lo16(ce.x) * S;
      const float* g1 = gw_s + hi16(ce.x) * S;
      const float* g2 = gw_s + lo16(ce.y) * S;
      const float4 q = *reinterpret_cast<const float4*>(pt.own_w + 4 * (size_t)c);
      const float* wc = w_s + it * Sn;  // wc[lv + 1]: half level k0 + lv
#pragma unroll
      for (int j = 0; j < L / 4; ++j) {
        const int lv = l0 + j, k = k0 + lv;
        if (k > nlev) break;
        float r = 0.0f;
        if (k > 0 && k < nlev) {
          const float h = fmat(q.z, g2[lv], fmat(q.y, g1[lv], q.x * g0[lv]));
          const float wa = wc[lv + 1];
          r = fmat(-(wa * (wc[lv] - wc[lv + 2])), v.qdzh[k], -h);
        }
        dw_s[it * S + lv] = r;
      }
    }
    for (int i = threadIdx.x; i < nw4 * L; i += blockDim.x) {
      const int it = i / L, lv = i - it * L, k = k0 + lv;
      if (k < nlev) ddt_vn[(size_t)pt.e4_g[e4a + it] * nlev + k] = dv_s[it * S + lv];
    }
  }
}

// -------------------------------------------------------------------------
// A5 (predictor): Green-Gauss gradients of rho and theta_v (perturbations in
// mixed mode: the reference is horizontally uniform) in each cell's local
// frame: grad4 = (drho_x, drho_y, dth_x, dth_y) as 4 planes [4][nc*nlev].
// -------------------------------------------------------------------------
// exner_ref_c: the per-column reference exner over terrain (kTerr).
template <class T, bool kTerr = false>
__global__ void sn_cell_grad(GridT<T> g, VertT<T> v, const T* __restrict__ rho, const T* __restrict__ theta,
                             T* __restrict__ grad4, const double* __restrict__ exner,
                             const double* __restrict__ exner_pr, double exfac, double* __restrict__ pex,
                             const double* __restrict__ exner_ref_c) {
  int c, k;
  const int nlev = v.nlev;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const size_t n = (size_t)g.nc * nlev;
  const int* cc = g.c2e2c + 3 * (size_t)c;
  const T* G = g.grad_c + 6 * (size_t)c;
  const size_t i = (size_t)c * nlev + k;
  const double ex_ref = kTerr ? exner_ref_c[i] : v.exner_ref[k];
  // extrapolated exner perturbation (1 + a) pr - a pr_old of this cell, for the
  // pressure gradient at its edges: FP64, or a double-word pair in mixed mode
  // (exner is near 1, the difference across an edge ~1e-5 of it)
  if constexpr (kMixed<T>) {
    const df a = to_df(1.0 + exfac), b = to_df(exfac);
    reinterpret_cast<df*>(pex)[i] = a * (to_df(exner[i]) - to_df(ex_ref)) - b * to_df(exner_pr[i]);
  } else {
    pex[i] = (1.0 + exfac) * (exner[i] - ex_ref) - exfac * exner_pr[i];
  }
  const size_t i0 = (size_t)cc[0] * nlev + k, i1 = (size_t)cc[1] * nlev + k, i2 = (size_t)cc[2] * nlev + k;
  const T r = rho[i], t = theta[i];
  if constexpr (kMixed<T>) {
    const T r0 = rho[i0] - r, r1 = rho[i1] - r, r2 = rho[i2] - r;
    const T t0 = theta[i0] - t, t1 = theta[i1] - t, t2 = theta[i2] - t;
    grad4[i] = G[0] * r0 + G[2] * r1 + G[4] * r2;
    grad4[n + i] = G[1] * r0 + G[3] * r1 + G[5] * r2;
    grad4[2 * n + i] = G[0] * t0 + G[2] * t1 + G[4] * t2;
    grad4[3 * n + i] = G[1] * t0 + G[3] * t1 + G[5] * t2;
  } else {
    // sum G_j psi_j - (sum G_j) psi_c: four FP64 operations per component
    // instead of the differences' shared three plus three (the gradient only
    // moves the upwind value by a small fraction of it, so the cancellation
    // is harmless)
    const T* S = g.grad_s + 2 * (size_t)c;
    const T r0 = rho[i0], r1 = rho[i1], r2 = rho[i2];
    const T t0 = theta[i0], t1 = theta[i1], t2 = theta[i2];
    grad4[i] = fmat(G[4], r2, fmat(G[2], r1, fmat(G[0], r0, -(S[0] * r))));
    grad4[n + i] = fmat(G[5], r2, fmat(G[3], r1, fmat(G[1], r0, -(S[1] * r))));
    grad4[2 * n + i] = fmat(G[4], t2, fmat(G[2], t1, fmat(G[0], t0, -(S[0] * t))));
    grad4[3 * n + i] = fmat(G[5], t2, fmat(G[3], t1, fmat(G[1], t0, -(S[1] * t))));
  }
}

// -------------------------------------------------------------------------
// A6 (predictor edges): upwind rho_e/theta_e from the back trajectory over
// dt/2, horizontal pressure gradient with the extrapolated exner perturbation,
// and the vn predictor.  FP64 mode reads totals; mixed mode reads the
// perturbations of rho and theta_v and adds the reference back.  The
// extrapolated exner perturbations come per cell from sn_cell_grad; their
// difference across the edge is taken in FP64 (double-word FP32 in mixed
// mode): neighbouring perturbations agree to 4-5 digits, more than FP32 carries.
// -------------------------------------------------------------------------
// Over terrain (kTerr) the pressure gradient is taken along the true
// horizontal: the along-level difference minus the slope of the full level
// times the edge mean of the two cells' vertical derivatives (centred, one-
// sided at the top and the ground) of the extrapolated exner perturbation.
template <class T, bool kTerr = false>
__global__ void sn_edge_pred(GridT<T> g, VertT<T> v, ScalT<T> sc, const T* __restrict__ vn,
                             const T* __restrict__ vt, const T* __restrict__ ddt_vn, const T* __restrict__ rho,
                             const T* __restrict__ theta, const double* __restrict__ pex,
                             const double* __restrict__ cid64, const T* __restrict__ grad4, T* __restrict__ rho_e,
                             T* __restrict__ theta_e,
                             T* __restrict__ hpg, T* __restrict__ vn_p, TerrT<T> tr) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t n = (size_t)g.nc * nlev;
  const size_t ie = (size_t)e * nlev + k;
  const T vne = vn[ie], vte = vt[ie];
  const int side = vne >= T(0) ? 0 : 1;
  const int cu = g.e2c[2 * e + side];
  // offset of the back-trajectory point from the upwind cell's centre, with
  // the half substep folded into the stored normal and tangent: two FMAs each
  const T* u = g.upw_s + 12 * (size_t)e + 6 * side;
  const T dx = fmat(-vne, u[2], fmat(-vte, u[4], u[0]));
  const T dy = fmat(-vne, u[3], fmat(-vte, u[5], u[1]));
  const size_t iu = (size_t)cu * nlev + k;
  T ru = rho[iu], tu = theta[iu];
  if constexpr (kMixed<T>) {
    ru += v.rho_ref[k];
    tu += v.theta_ref[k];
  }
  const T re = fmat(grad4[iu], dx, fmat(grad4[n + iu], dy, ru));
  const T te = fmat(grad4[2 * n + iu], dx, fmat(grad4[3 * n + iu], dy, tu));
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const size_t i0 = (size_t)c0 * nlev + k, i1 = (size_t)c1 * nlev + k;
  // cpd theta_e d(pr)/dn with cpd folded into the edge factor cpd / d_e (and,
  // over terrain, into the stored slope)
  T h;
  const int km = k > 0 ? k - 1 : 0, kp = k + 1 < nlev ? k + 1 : nlev - 1;
  if constexpr (kMixed<T>) {
    const df* p = reinterpret_cast<const df*>(pex);
    if constexpr (kTerr) {
      const size_t b0 = (size_t)c0 * nlev, b1 = (size_t)c1 * nlev;
      const T dz0 = to_float(p[b0 + km] - p[b0 + kp]) * tr.inv_dzm_c[i0];
      const T dz1 = to_float(p[b1 + km] - p[b1 + kp]) * tr.inv_dzm_c[i1];
      h = te * (to_float(p[i1] - p[i0]) * g.cpd_inv_d[e] - tr.ddxn_mc[ie] * (T(0.5) * (dz0 + dz1)));
    } else {
      h = te * (to_float(p[i1] - p[i0]) * g.cpd_inv_d[e]);
    }
  } else {
    if constexpr (kTerr) {
      const size_t b0 = (size_t)c0 * nlev, b1 = (size_t)c1 * nlev;
      const double dz0 = (pex[b0 + km] - pex[b0 + kp]) * tr.inv_dzm_c[i0];
      const double dz1 = (pex[b1 + km] - pex[b1 + kp]) * tr.inv_dzm_c[i1];
      h = te * (T)((pex[i1] - pex[i0]) * cid64[e] - tr.ddxn_mc[ie] * (0.5 * (dz0 + dz1)));
    } else {
      h = te * (T)((pex[i1] - pex[i0]) * cid64[e]);
    }
  }
  rho_e[ie] = re;
  theta_e[ie] = te;
  hpg[ie] = h;
  vn_p[ie] = vne + sc.dt_s * (ddt_vn[ie] - h);
}

// -------------------------------------------------------------------------
// A6 over steep terrain: at the listed edge levels the pressure gradient is
// taken at the edge's height, each cell's total exner (extrapolated
// perturbation plus the column's reference) interpolated there by the
// quadratic through three of its levels; the predictor's vn at those points
// follows.  Runs after sn_edge_pred, over the listed points only.
// -------------------------------------------------------------------------
template <class T>
__global__ void sn_edge_hpg_steep(GridT<T> g, VertT<T> v, ScalT<T> sc, int n, const int* __restrict__ idx,
                                  const double* __restrict__ wts, const double* __restrict__ pex,
                                  const double* __restrict__ exref_c, const double* __restrict__ cid64,
                                  const T* __restrict__ theta_e, const T* __restrict__ vn,
                                  const T* __restrict__ ddt_vn, T* __restrict__ hpg, T* __restrict__ vn_p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nlev = v.nlev;
  const int e = idx[4 * i], k = idx[4 * i + 1];
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const size_t b0 = (size_t)c0 * nlev + idx[4 * i + 2], b1 = (size_t)c1 * nlev + idx[4 * i + 3];
  const double* w = wts + 6 * (size_t)i;
  const size_t ie = (size_t)e * nlev + k;
  T h;
  if constexpr (kMixed<T>) {
    const df* p = reinterpret_cast<const df*>(pex);
    df s0{0.f, 0.f}, s1{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s0 = s0 + to_df(w[j]) * (p[b0 + j] + to_df(exref_c[b0 + j]));
      s1 = s1 + to_df(w[3 + j]) * (p[b1 + j] + to_df(exref_c[b1 + j]));
    }
    h = theta_e[ie] * (to_float(s1 - s0) * g.cpd_inv_d[e]);
  } else {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s0 = fma(w[j], pex[b0 + j] + exref_c[b0 + j], s0);
      s1 = fma(w[3 + j], pex[b1 + j] + exref_c[b1 + j], s1);
    }
    h = theta_e[ie] * (T)((s1 - s0) * cid64[e]);
  }
  hpg[ie] = h;
  vn_p[ie] = vn[ie] + sc.dt_s * (ddt_vn[ie] - h);
}

// -------------------------------------------------------------------------
// A8 + A9 (corrector edges): vn corrector with time-weighted advective
// tendencies, the predictor's pressure gradient and fourth-order divergence
// damping; the increment is formed in T, the update in FP64 (in place).
// -------------------------------------------------------------------------
// Both tile shapes update every (edge, level) with sn_edge_corr_at.
template <class T>
__device__ __forceinline__ void sn_edge_corr_at(const ScalT<T>& sc, size_t ie, T ddamp, T d0k, T d1k,
                                                double* vn, const T* ddt_vn0, const T* ddt_vn1, const T* hpg,
                                                float* m_vn) {
  // fourth-order divergence damping: divdamp_fac Abar^2 grad_n(dd2), coefficient per edge
  const T damp = ddamp * (d1k - d0k);
  const T tend = fmat(sc.wnow_vel, ddt_vn0[ie], fmat(sc.wnew_vel, ddt_vn1[ie], -hpg[ie]));
  const T inc = fmat(sc.dt_s, tend, -damp);
  if constexpr (kMixed<T>) {
    const double vnn = vn[ie] + f2d(inc);
    vn[ie] = vnn;
    m_vn[ie] = d2f(vnn);
  } else {
    vn[ie] = vn[ie] + (double)inc;
  }
}

template <class T>
__global__ void sn_edge_corr(GridT<T> g, VertT<T> v, ScalT<T> sc, double* __restrict__ vn,
                             const T* __restrict__ ddt_vn0, const T* __restrict__ ddt_vn1,
                             const T* __restrict__ hpg, const T* __restrict__ divd2, float* __restrict__ m_vn,
                             int shape) {
  const int nlev = v.nlev;
  if (shape) {  // one warp per edge, its lanes over the levels
    const int e = warp_point();
    if (e >= g.ne) return;
    const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
    const T ddamp = g.ddamp_e[e];
    const T* d0 = divd2 + (size_t)c0 * nlev;
    const T* d1 = divd2 + (size_t)c1 * nlev;
    for (int k = lane_id(); k < nlev; k += 32)
      sn_edge_corr_at(sc, (size_t)e * nlev + k, ddamp, d0[k], d1[k], vn, ddt_vn0, ddt_vn1, hpg, m_vn);
    return;
  }
  int e, k;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  sn_edge_corr_at(sc, (size_t)e * nlev + k, g.ddamp_e[e], divd2[(size_t)c0 * nlev + k],
                  divd2[(size_t)c1 * nlev + k], vn, ddt_vn0, ddt_vn1, hpg, m_vn);
}

// -------------------------------------------------------------------------
// Cell divergence D = (1/A_c) sum_e s l_e vn_e of vn* (fourth-order damping and
// flux filter of the predictor) or vn^{n+1} (flux filter of the corrector).
// The predictor launch also updates the exner extrapolation history,
// exner_pr = exner - exner_ref (sn_edge_pred, its last reader, has completed).
// Both tile shapes evaluate every (cell, level) with the same FMAs.
// -------------------------------------------------------------------------
template <class T, bool kTerr = false>
__global__ void sn_cell_div(GridT<T> g, VertT<T> v, const T* __restrict__ vn, T* __restrict__ divd,
                            const double* __restrict__ exner, double* __restrict__ exner_pr,
                            const double* __restrict__ exner_ref_c, int shape) {
  const int nlev = v.nlev;
  if (shape) {  // one warp per cell, its lanes over the levels
    const int c = warp_point();
    if (c >= g.nc) return;
    const int* ce = g.c2e + 3 * (size_t)c;
    const T* dvp = g.div_c + 3 * (size_t)c;
    const T dv0 = dvp[0], dv1 = dvp[1], dv2 = dvp[2];
    const T* x0 = vn + (size_t)ce[0] * nlev;
    const T* x1 = vn + (size_t)ce[1] * nlev;
    const T* x2 = vn + (size_t)ce[2] * nlev;
    for (int k = lane_id(); k < nlev; k += 32) {
      const size_t i = (size_t)c * nlev + k;
      divd[i] = fmat(dv2, x2[k], fmat(dv1, x1[k], dv0 * x0[k]));
      if (exner_pr) exner_pr[i] = exner[i] - (kTerr ? exner_ref_c[i] : v.exner_ref[k]);
    }
    return;
  }
  int c, k;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const int* ce = g.c2e + 3 * (size_t)c;
  const T* dv = g.div_c + 3 * (size_t)c;
  const size_t i = (size_t)c * nlev + k;
  divd[i] = fmat(dv[2], vn[(size_t)ce[2] * nlev + k], fmat(dv[1], vn[(size_t)ce[1] * nlev + k],
                                                           dv[0] * vn[(size_t)ce[0] * nlev + k]));
  if (exner_pr) exner_pr[i] = exner[i] - (kTerr ? exner_ref_c[i] : v.exner_ref[k]);
}

// -------------------------------------------------------------------------
// Divergences of the horizontal mass and theta fluxes with the flux-velocity
// filter, per cell and level, summed in FP64 (double-word FP32 in mixed
// mode, stored as the pair):
//   vf_e = vn_e + divflux (D_c1 - D_c0)/d_e,  F_e = rho_e vf_e,
//   div_m = sum s l F / A,  div_t = sum s l F theta_e / A
// -------------------------------------------------------------------------
// Over terrain (kTerr) each flux carries its edge layer thickness over the
// cell's, fx_ratio = dz_e / dz_c: div_m = (1/dz_c) sum s l F dz_e / A.
template <class T, bool kTerr = false>
__global__ void sn_cell_fluxdiv(GridT<T> g, VertT<T> v, ScalT<T> sc, const T* __restrict__ vn,
                                const T* __restrict__ divd, const T* __restrict__ rho_e,
                                const T* __restrict__ theta_e, const double* __restrict__ div_c64,
                                double* __restrict__ div_m, double* __restrict__ div_t,
                                const T* __restrict__ fx_ratio) {
  const int nlev = v.nlev;
  if constexpr (kMixed<T>) {
    // FP32 fluxes, sums in double-word FP32: FP64-grade accumulation (mass
    // conserved to about 2^-48 of the flux) without the slow FP64 pipe.  One
    // warp per cell: the cell's three edges, their filter coefficients and
    // the divergence rows of their cells are loaded once.
    const int c = warp_point();
    if (c >= g.nc) return;
    const int* ce = g.c2e + 3 * (size_t)c;
    size_t be[3], bd0[3], bd1[3];
    T fd[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int e = ce[j];
      be[j] = (size_t)e * nlev;
      bd0[j] = (size_t)g.e2c[2 * e] * nlev;
      bd1[j] = (size_t)g.e2c[2 * e + 1] * nlev;
      fd[j] = g.fdiv_e[e];
    }
    const df* dvp = reinterpret_cast<const df*>(g.div_c_hl) + 3 * (size_t)c;
    const df dv[3] = {dvp[0], dvp[1], dvp[2]};
    for (int k = lane_id(); k < nlev; k += 32) {
      df dm{0.f, 0.f}, dt{0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const size_t ie = be[j] + k;
        const T vf = vn[ie] + fd[j] * (divd[bd1[j] + k] - divd[bd0[j] + k]);
        T f = rho_e[ie] * vf;
        if constexpr (kTerr) f = f * fx_ratio[((size_t)c * 3 + j) * nlev + k];
        const T ft = f * theta_e[ie];
        const df w = dv[j];
        dm = dm + w * f;
        dt = dt + w * ft;
      }
      // stored as the double-word pair itself (8 bytes, read by the column solve)
      reinterpret_cast<df*>(div_m)[(size_t)c * nlev + k] = dm;
      reinterpret_cast<df*>(div_t)[(size_t)c * nlev + k] = dt;
    }
  } else {
    int c, k;
    if (!flat_index(g.nc, nlev, c, k)) return;
    const int* ce = g.c2e + 3 * (size_t)c;
    const double* dv = div_c64 + 3 * (size_t)c;
    double dm = 0.0, dt = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int e = ce[j];
      const size_t ie = (size_t)e * nlev + k;
      const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
      const T vf = vn[ie] + g.fdiv_e[e] * (divd[(size_t)c1 * nlev + k] - divd[(size_t)c0 * nlev + k]);
      T f = rho_e[ie] * vf;
      if constexpr (kTerr) f = f * fx_ratio[((size_t)c * 3 + j) * nlev + k];
      const T ft = f * theta_e[ie];
      dm += dv[j] * (double)f;
      dt += dv[j] * (double)ft;
    }
    div_m[(size_t)c * nlev + k] = dm;
    div_t[(size_t)c * nlev + k] = dt;
  }
}

// -------------------------------------------------------------------------
// FP64 mode: the same divergences from fluxes computed once per edge (the
// cell form above computes each edge's flux once for each of its two cells,
// and the FP64 mode is bound by the FP64 issue rate):
//   sn_edge_flux:    F_e = rho_e vf_e, Ft_e = F_e theta_e (edges, full levels)
//   sn_cell_fluxsum: div_m = sum s l F / A, div_t = sum s l Ft / A, over
//                    terrain with each flux times dz_e / dz_c
// -------------------------------------------------------------------------
__global__ void sn_edge_flux(GridT<double> g, VertT<double> v, const double* __restrict__ vn,
                             const double* __restrict__ divd, const double* __restrict__ rho_e,
                             const double* __restrict__ theta_e, double* __restrict__ flx_m,
                             double* __restrict__ flx_t) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t ie = (size_t)e * nlev + k;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const double vf = fma(g.fdiv_e[e], divd[(size_t)c1 * nlev + k] - divd[(size_t)c0 * nlev + k], vn[ie]);
  const double f = rho_e[ie] * vf;
  flx_m[ie] = f;
  flx_t[ie] = f * theta_e[ie];
}

template <bool kTerr>
__global__ void sn_cell_fluxsum(GridT<double> g, VertT<double> v, const double* __restrict__ flx_m,
                                const double* __restrict__ flx_t, double* __restrict__ div_m,
                                double* __restrict__ div_t, const double* __restrict__ fx_ratio) {
  int c, k;
  const int nlev = v.nlev;
  if (!flat_index(g.nc, nlev, c, k)) return;
  const int* ce = g.c2e + 3 * (size_t)c;
  const double* dv = g.div_c + 3 * (size_t)c;
  double dm = 0.0, dt = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const size_t ie = (size_t)ce[j] * nlev + k;
    double fm = flx_m[ie], ft = flx_t[ie];
    if constexpr (kTerr) {
      const double r = fx_ratio[((size_t)c * 3 + j) * nlev + k];
      fm = fm * r;
      ft = ft * r;
    }
    dm = fma(dv[j], fm, dm);
    dt = fma(dv[j], ft, dt);
  }
  div_m[(size_t)c * nlev + k] = dm;
  div_t[(size_t)c * nlev + k] = dt;
}

// -------------------------------------------------------------------------
// Mixed mode: FP32 mirrors of the FP64 state at the start of a call
// (the caller may have changed the state between calls).  One launch over
// ne*nlev + nc*(nlev+1).
// -------------------------------------------------------------------------
__global__ void mx_refresh(int ne, int nc, int nlev, const double* __restrict__ exner_ref,
                           const double* __restrict__ theta_ref, const double* __restrict__ rho_ref, StateView st,
                           Mirrors m) {
  const int nlevp = nlev + 1;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nedge = (unsigned)ne * nlev;
  if (i < nedge) {
    m.vn[i] = d2f(st.vn[i]);
    return;
  }
  i -= nedge;
  if (i >= (unsigned)nc * nlevp) return;
  const int c = (int)(i / (unsigned)nlevp), k = (int)(i - (unsigned)c * nlevp);
  m.w[i] = d2f(st.w[i]);
  if (k < nlev) {
    const size_t j = (size_t)c * nlev + k;
    m.rho[j] = d2f(st.rho[j] - rho_ref[k]);
    m.th[j] = d2f(st.theta_v[j] - theta_ref[k]);
  }
}

// -------------------------------------------------------------------------
// A10 diffusion
// -------------------------------------------------------------------------
// cells: div vn; vertices: curl vn and the vertex velocity (xyz)
template <class T>
__global__ void diff_div_curl_uv(GridT<T> g, VertT<T> v, const T* __restrict__ vn, T* __restrict__ div_vn,
                                 T* __restrict__ zeta, T* __restrict__ uv3) {
  const int nlev = v.nlev;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlev;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)c * nlev);
    const int* ce = g.c2e + 3 * (size_t)c;
    const T* dv = g.div_c + 3 * (size_t)c;
    div_vn[i] = dv[0] * vn[(size_t)ce[0] * nlev + k] + dv[1] * vn[(size_t)ce[1] * nlev + k] +
                dv[2] * vn[(size_t)ce[2] * nlev + k];
    return;
  }
  i -= ncell;
  const size_t nvl = (size_t)g.nv * nlev;
  if (i >= nvl) return;
  int vx = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)vx * nlev);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const T* cw = g.curl_v + 6 * (size_t)vx;
  const T* U = g.uv_w + 18 * (size_t)vx;
  T z = 0, ux = 0, uy = 0, uz = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const T x = vn[(size_t)ve[j] * nlev + k];
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
template <class T>
__global__ void diff_edge_smag(GridT<T> g, VertT<T> v, const T* __restrict__ div_vn, const T* __restrict__ zeta,
                               const T* __restrict__ uv3, T* __restrict__ nu, T* __restrict__ lap) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t nvl = (size_t)g.nv * nlev;
  const int* dm = g.e2c2v + 4 * (size_t)e;
  const size_t im = (size_t)dm[0] * nlev + k, ip = (size_t)dm[1] * nlev + k;
  const size_t i2 = (size_t)dm[2] * nlev + k, i3 = (size_t)dm[3] * nlev + k;
  const T* nt = g.nt + 6 * (size_t)e;
  const T dtx = uv3[ip] - uv3[im], dty = uv3[nvl + ip] - uv3[nvl + im], dtz = uv3[2 * nvl + ip] - uv3[2 * nvl + im];
  const T dnx = uv3[i3] - uv3[i2], dny = uv3[nvl + i3] - uv3[nvl + i2], dnz = uv3[2 * nvl + i3] - uv3[2 * nvl + i2];
  const T il = g.inv_l[e], idn = g.inv_dn[e];
  const T tension = (dnx * nt[0] + dny * nt[1] + dnz * nt[2]) * idn - (dtx * nt[3] + dty * nt[4] + dtz * nt[5]) * il;
  const T shear = (dtx * nt[0] + dty * nt[1] + dtz * nt[2]) * il + (dnx * nt[3] + dny * nt[4] + dnz * nt[5]) * idn;
  const size_t ie = (size_t)e * nlev + k;
  nu[ie] = g.smag_a[e] * sqrt(tension * tension + shear * shear);
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  lap[ie] = (div_vn[(size_t)c1 * nlev + k] - div_vn[(size_t)c0 * nlev + k]) * g.inv_d[e] -
            (zeta[ip] - zeta[im]) * il;
}

// cells (half-level range): div of lap vn, cell Laplacian of w, theta increment;
// vertices: curl of lap vn
template <class T>
__global__ void diff_second(GridT<T> g, VertT<T> v, ScalT<T> sc, const T* __restrict__ lap, const T* __restrict__ nu,
                            const T* __restrict__ w, const T* __restrict__ theta, T* __restrict__ div_l,
                            T* __restrict__ lap_w, T* __restrict__ dtheta, T* __restrict__ curl_l,
                            const T* __restrict__ tenh_ex) {
  const int nlev = v.nlev, nlevp = nlev + 1;
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ncell = (unsigned)g.nc * nlevp;
  if (i < ncell) {
    int c = (int)(i / (unsigned)nlevp), k = (int)(i - (unsigned)c * nlevp);
    const int* ce = g.c2e + 3 * (size_t)c;
    const int* cc = g.c2e2c + 3 * (size_t)c;
    const T* L = g.lap_c + 3 * (size_t)c;
    const T wc = w[(size_t)c * nlevp + k];
    T lw = L[0] * (w[(size_t)cc[0] * nlevp + k] - wc);
    lw += L[1] * (w[(size_t)cc[1] * nlevp + k] - wc);
    lw += L[2] * (w[(size_t)cc[2] * nlevp + k] - wc);
    lap_w[i] = lw;
    if (k < nlev) {
      const T* dv = g.div_c + 3 * (size_t)c;
      const size_t ic = (size_t)c * nlev + k;
      div_l[ic] = dv[0] * lap[(size_t)ce[0] * nlev + k] + dv[1] * lap[(size_t)ce[1] * nlev + k] +
                  dv[2] * lap[(size_t)ce[2] * nlev + k];
      if (sc.hdiff_temp) {
        const T tc = theta[ic];
        T n0 = nu[(size_t)ce[0] * nlev + k], n1 = nu[(size_t)ce[1] * nlev + k], n2 = nu[(size_t)ce[2] * nlev + k];
        if (k >= nlev - sc.tenh_levels) {
          // enhanced near-surface temperature diffusion: the edge coefficient
          // raised by fac A_e / dtime max(e_c, e_nbr)
          const T ex = tenh_ex[ic];
          n0 += g.tenh_a[ce[0]] * max(ex, tenh_ex[(size_t)cc[0] * nlev + k]);
          n1 += g.tenh_a[ce[1]] * max(ex, tenh_ex[(size_t)cc[1] * nlev + k]);
          n2 += g.tenh_a[ce[2]] * max(ex, tenh_ex[(size_t)cc[2] * nlev + k]);
        }
        T f = L[0] * n0 * (theta[(size_t)cc[0] * nlev + k] - tc);
        f += L[1] * n1 * (theta[(size_t)cc[1] * nlev + k] - tc);
        f += L[2] * n2 * (theta[(size_t)cc[2] * nlev + k] - tc);
        dtheta[ic] = sc.dtime * f;
      }
    }
    return;
  }
  i -= ncell;
  if (i >= (unsigned)g.nv * nlev) return;
  int vx = (int)(i / (unsigned)nlev), k = (int)(i - (unsigned)vx * nlev);
  const int* ve = g.v2e + 6 * (size_t)vx;
  const T* cw = g.curl_v + 6 * (size_t)vx;
  T z = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) z += cw[j] * lap[(size_t)ve[j] * nlev + k];
  curl_l[i] = z;
}

// cells, the lowest tenh_levels levels: the excess factor of the enhanced
// temperature diffusion, e_c = min(1, (|theta_c - mean of the three neighbours|
// - thresh) / thresh) where above the threshold, else 0 (theta as the stencil
// views it: the FP64 state, or the mixed mode's perturbation from a per-level
// offset, which the difference does not see)
template <class T>
__global__ void diff_tenh_excess(GridT<T> g, VertT<T> v, ScalT<T> sc, const T* __restrict__ theta,
                                 T* __restrict__ ex) {
  const int nlev = v.nlev, nl = sc.tenh_levels;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (unsigned)g.nc * (unsigned)nl) return;
  const int c = (int)(i / (unsigned)nl), k = nlev - nl + (int)(i - (unsigned)c * (unsigned)nl);
  const int* cc = g.c2e2c + 3 * (size_t)c;
  const size_t ic = (size_t)c * nlev + k;
  const T nbr = (theta[(size_t)cc[0] * nlev + k] + theta[(size_t)cc[1] * nlev + k] + theta[(size_t)cc[2] * nlev + k]) /
                T(3);
  const T x = (abs(theta[ic] - nbr) - sc.tenh_thresh) / sc.tenh_thresh;
  ex[ic] = x < T(0) ? T(0) : (x > T(1) ? T(1) : x);
}

// edges: vn update (FP64, in place)
template <class T>
__global__ void diff_edge_update(GridT<T> g, VertT<T> v, ScalT<T> sc, double* __restrict__ vn,
                                 const T* __restrict__ nu, const T* __restrict__ lap, const T* __restrict__ div_l,
                                 const T* __restrict__ curl_l, float* __restrict__ m_vn) {
  int e, k;
  const int nlev = v.nlev;
  if (!flat_index(g.ne, nlev, e, k)) return;
  const size_t ie = (size_t)e * nlev + k;
  const int c0 = g.e2c[2 * e], c1 = g.e2c[2 * e + 1];
  const int vm = g.e2v[2 * e], vp = g.e2v[2 * e + 1];
  const T lap2 = (div_l[(size_t)c1 * nlev + k] - div_l[(size_t)c0 * nlev + k]) * g.inv_d[e] -
                 (curl_l[(size_t)vp * nlev + k] - curl_l[(size_t)vm * nlev + k]) * g.inv_l[e];
  const T inc = sc.dtime * nu[ie] * lap[ie] - g.k4_a[e] * lap2;
  if constexpr (kMixed<T>) {
    const double vnn = vn[ie] + f2d(inc);
    vn[ie] = vnn;
    m_vn[ie] = d2f(vnn);
  } else {
    vn[ie] = vn[ie] + (double)inc;
  }
}

// cells (half-level range): w fourth-order diffusion, theta/exner update (FP64, in place)
template <class T>
__global__ void diff_cell_update(GridT<T> g, VertT<T> v, ScalT<T> sc, const double* __restrict__ theta_ref,
                                 const double* __restrict__ exner_ref, double rd_o_cvd, StateView st,
                                 const T* __restrict__ lap_w, const T* __restrict__ dtheta, Mirrors m) {
  int c, k;
  const int nlev = v.nlev, nlevp = nlev + 1;
  if (!flat_index(g.nc, nlevp, c, k)) return;
  if (k > 0 && k < nlev) {
    const int* cc = g.c2e2c + 3 * (size_t)c;
    const T* L = g.lap_c + 3 * (size_t)c;
    const T lc = lap_w[(size_t)c * nlevp + k];
    T l2 = L[0] * (lap_w[(size_t)cc[0] * nlevp + k] - lc);
    l2 += L[1] * (lap_w[(size_t)cc[1] * nlevp + k] - lc);
    l2 += L[2] * (lap_w[(size_t)cc[2] * nlevp + k] - lc);
    const size_t iw = (size_t)c * nlevp + k;
    if constexpr (kMixed<T>) {
      const double wn = st.w[iw] - f2d(g.k4w_c[c] * l2);
      st.w[iw] = wn;
      m.w[iw] = d2f(wn);
    } else {
      st.w[iw] = st.w[iw] - (double)(g.k4w_c[c] * l2);
    }
  }
  if (k < nlev && sc.hdiff_temp) {
    const size_t ic = (size_t)c * nlev + k;
    const double th = st.theta_v[ic];
    if constexpr (kMixed<T>) {
      // exner (1 + rd/cvd dtheta/theta): the FP32 increment of a value near 1
      const float dth = dtheta[ic];
      const double thn = th + f2d(dth);
      st.theta_v[ic] = thn;
      st.exner[ic] = st.exner[ic] + f2d(d2f(st.exner[ic]) * ((float)rd_o_cvd * dth / d2f(th)));
      m.th[ic] = d2f(thn - theta_ref[k]);
    } else {
      const double thn = th + (double)dtheta[ic];
      const double exn = st.exner[ic] * (1.0 + rd_o_cvd * (thn - th) / th);
      st.theta_v[ic] = thn;
      st.exner[ic] = exn;
    }
  }
}

}  // namespace

// -------------------------------------------------------------------------
// launch sequences
// -------------------------------------------------------------------------
template <class T>
void launch_velocity_tendencies(const Ctx<T>& x, const T* vn, const T* w, T* ddt_vn, T* ddt_w, const T* divd,
                                T* divd2, cudaStream_t s, const int* threads, T* wcc, const int* shapes) {
  const GridT<T>& g = x.g;
  const VertT<T>& v = x.v;
  const WorkT<T>& wk = x.w;
  const TerrT<T>& tr = x.tr;
  const int nlev = v.nlev, nlevp = nlev + 1;
  const bool terr = tr.wgt_e != nullptr && wcc != nullptr;
  if constexpr (kMixed<T>) {
    if (x.vp.n_patches > 0 && !terr) {  // rows A1-A4 in one launch
      const VaPatchT& pt = x.vp;
      const size_t smem =
          va_fused_smem_floats(pt.max_e0, pt.max_e1, pt.max_c3, pt.max_c0, pt.max_v3, pt.max_e4) * sizeof(float);
      ICON_LAUNCH_SMEM("va_fused_f32", (unsigned)pt.n_patches, kVaThreads, smem, s, va_fused, g, v, pt, vn, w, wk.vt,
                       ddt_vn, ddt_w, divd, divd2);
      return;
    }
  }
  ICON_LAUNCH(kname<T>("va_edge_pre", "va_edge_pre_f32"), blocks_by_shape(SH(0), g.ne, nlev, TH(0)), TH(0), s,
              va_edge_pre<T>, g, v, vn, wk.vt, wk.ekin_e, wk.vn_ie, terr ? tr.wgt_e : nullptr, SH(0));
  if (terr)
    ICON_LAUNCH(kname<T>("va_concorr", "va_concorr_f32"), blocks_for((long long)g.nc * nlevp, TH(14)), TH(14), s,
                va_concorr<T>, g, v, tr, wk.vn_ie, wk.vt, wcc);
  const long long n2 = (long long)g.nc * nlev + (long long)g.nv * nlevp;
  ICON_LAUNCH(kname<T>("va_cell_vert", "va_cell_vert_f32"), blocks_for(n2, TH(1)), TH(1), s, va_cell_vert<T>, g,
              v, vn, w, wk.ekin_e, wk.ekin_c, divd, divd2, wk.zeta, wk.w_v, wk.wq, terr ? (const T*)wcc : nullptr);
  if (terr) {
    ICON_LAUNCH(kname<T>("va_edge_tend_terrain", "va_edge_tend_terrain_f32"),
                blocks_for((long long)g.ne * nlevp, TH(2)), TH(2), s, (va_edge_tend<T, true>), g, v, wk.vn_ie, w, wk.vt,
                wk.ekin_c, wk.zeta, wk.w_v, ddt_vn, wk.gw_e, tr, (const T*)wk.wq);
    ICON_LAUNCH(kname<T>("va_cell_w_terrain", "va_cell_w_terrain_f32"), blocks_by_shape(SH(3), g.nc, nlevp, TH(3)),
                TH(3), s, (va_cell_w<T, true>), g, v, w, wk.gw_e, ddt_w, tr, wcc, SH(3));
  } else {
    ICON_LAUNCH(kname<T>("va_edge_tend", "va_edge_tend_f32"), blocks_for((long long)g.ne * nlevp, TH(2)), TH(2),
                s, (va_edge_tend<T, false>), g, v, wk.vn_ie, w, wk.vt, wk.ekin_c, wk.zeta, wk.w_v, ddt_vn, wk.gw_e, tr,
                (const T*)wk.wq);
    ICON_LAUNCH(kname<T>("va_cell_w", "va_cell_w_f32"), blocks_by_shape(SH(3), g.nc, nlevp, TH(3)), TH(3), s,
                (va_cell_w<T, false>), g, v, w, wk.gw_e, ddt_w, tr, wcc, SH(3));
  }
}

// Flux divergences of the mass and theta fluxes of the velocity vn (with the
// flux filter): the mixed mode sums FP32 fluxes per cell in double-word
// arithmetic; the FP64 mode computes each edge's fluxes once, then sums them.
template <class T, bool kTerr>
void launch_fluxdiv(const Engine& en, const Ctx<T>& x, const T* vn, const char* name, cudaStream_t s) {
  const int* threads = en.threads;
  const GridT<T>& g = x.g;
  const VertT<T>& v = x.v;
  const WorkT<T>& wk = x.w;
  const int nlev = v.nlev;
  if constexpr (kMixed<T>) {
    ICON_LAUNCH(name, blocks_by_point<T>(g.nc, nlev, TH(7)), TH(7), s, (sn_cell_fluxdiv<T, kTerr>), g, v, x.s, vn,
                wk.divd, wk.rho_e, wk.theta_e, en.g64.div_c, en.wk.div_m, en.wk.div_t, x.tr.fx_ratio);
  } else {
    ICON_LAUNCH("sn_edge_flux", blocks_for((long long)g.ne * nlev, TH(15)), TH(15), s, sn_edge_flux, g, v, vn,
                wk.divd, wk.rho_e, wk.theta_e, wk.flx_m, wk.flx_t);
    ICON_LAUNCH(kTerr ? "sn_cell_fluxsum_terrain" : "sn_cell_fluxsum", blocks_for((long long)g.nc * nlev, TH(7)),
                TH(7), s, (sn_cell_fluxsum<kTerr>), g, v, wk.flx_m, wk.flx_t, en.wk.div_m, en.wk.div_t,
                x.tr.fx_ratio);
  }
}

// Rows A5-A9 of one substep; kTerr: the terrain forms, with the contravariant
// corrections of the predictor's and the corrector's winds in x.tr.wcc0/wcc1.
// s waits for event e: as an external event node when s is being captured
// into a graph (the wait then happens at every launch of the graph), else as
// a plain stream wait
void stream_wait_io(cudaStream_t s, cudaEvent_t e) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cudaStreamWaitEvent(s, e, cs == cudaStreamCaptureStatusActive ? cudaEventWaitExternal : 0);
}
void stream_record_io(cudaStream_t s, cudaEvent_t e) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0);
}

template <class T, bool kTerr>
void substep_impl(const Engine& en, const Ctx<T>& x, const StateView& st, cudaStream_t s) {
  const int* threads = en.threads;
  const int* shapes = en.shape;
  const GridT<T>& g = x.g;
  const VertT<T>& v = x.v;
  const WorkT<T>& wk = x.w;
  const TerrT<T>& tr = x.tr;
  const Mirrors& m = en.m;
  const int nlev = v.nlev;
  const long long nce = (long long)g.nc * nlev, nee = (long long)g.ne * nlev;
  const double* ex_ref_c = en.v.exner_ref_c;
  // stencil views of the state: the FP64 state itself, or the FP32 mirrors
  const T *s_vn, *s_w, *s_rho, *s_th, *s_wp;
  if constexpr (kMixed<T>) {
    s_vn = m.vn, s_w = m.w, s_rho = m.rho, s_th = m.th, s_wp = m.w_p;
  } else {
    s_vn = st.vn, s_w = st.w, s_rho = st.rho, s_th = st.theta_v, s_wp = en.wk.w_p;
  }
  const char* nm_grad = kTerr ? kname<T>("sn_cell_grad_terrain", "sn_cell_grad_terrain_f32")
                              : kname<T>("sn_cell_grad", "sn_cell_grad_f32");
  const char* nm_pred = kTerr ? kname<T>("sn_edge_pred_terrain", "sn_edge_pred_terrain_f32")
                              : kname<T>("sn_edge_pred", "sn_edge_pred_f32");
  const char* nm_div = kTerr ? kname<T>("sn_cell_div_terrain", "sn_cell_div_terrain_f32")
                             : kname<T>("sn_cell_div", "sn_cell_div_f32");
  const char* nm_flx = kTerr ? kname<T>("sn_cell_fluxdiv_terrain", "sn_cell_fluxdiv_terrain_f32")
                             : kname<T>("sn_cell_fluxdiv", "sn_cell_fluxdiv_f32");
  // ---------------- predictor ----------------
  launch_velocity_tendencies<T>(x, s_vn, s_w, wk.ddt_vn0, wk.ddt_w0, nullptr, nullptr, s, threads,
                                kTerr ? tr.wcc0 : nullptr, shapes);
  if (en.io_wait) stream_wait_io(s, en.io_wait);  // rho, theta_v, exner, exner_pr from here on
  ICON_LAUNCH(nm_grad, blocks_for(nce, TH(4)), TH(4), s, (sn_cell_grad<T, kTerr>), g, v, s_rho, s_th, wk.grad4,
              st.exner, st.exner_pr, en.sc.exfac, en.wk.pex, ex_ref_c);
  ICON_LAUNCH(nm_pred, blocks_for(nee, TH(5)), TH(5), s, (sn_edge_pred<T, kTerr>), g, v, x.s, s_vn, wk.vt,
              wk.ddt_vn0, s_rho, s_th, en.wk.pex, en.g64.cpd_inv_d, wk.grad4, wk.rho_e, wk.theta_e, wk.hpg, wk.vn_p, tr);
  if (kTerr && en.v.n_steep > 0)
    ICON_LAUNCH(kname<T>("sn_edge_hpg_steep", "sn_edge_hpg_steep_f32"), blocks_for(en.v.n_steep, 128), 128, s,
                sn_edge_hpg_steep<T>, g, v, x.s, en.v.n_steep, en.v.steep_idx, en.v.steep_w, en.wk.pex,
                en.v.exner_ref_c, en.g64.cpd_inv_d, wk.theta_e, s_vn, wk.ddt_vn0, wk.hpg, wk.vn_p);
  ICON_LAUNCH(nm_div, blocks_by_shape(SH(6), g.nc, nlev, TH(6)), TH(6), s, (sn_cell_div<T, kTerr>), g, v, wk.vn_p,
              wk.divd, st.exner, st.exner_pr, ex_ref_c, SH(6));
  launch_fluxdiv<T, kTerr>(en, x, wk.vn_p, nm_flx, s);
  if constexpr (kTerr)
    launch_column_terrain<T>(en, 0, st, wk.ddt_w0, wk.ddt_w1, tr.wcc0, s);
  else
    launch_column<T>(en, 0, st, wk.ddt_w0, wk.ddt_w1, s);
  // ---------------- corrector ----------------
  launch_velocity_tendencies<T>(x, wk.vn_p, s_wp, wk.ddt_vn1, wk.ddt_w1, wk.divd, wk.divd2, s, threads,
                                kTerr ? tr.wcc1 : nullptr, shapes);
  ICON_LAUNCH(kname<T>("sn_edge_corr", "sn_edge_corr_f32"), blocks_by_shape(SH(8), g.ne, nlev, TH(8)), TH(8), s,
              sn_edge_corr<T>, g, v, x.s, st.vn, wk.ddt_vn0, wk.ddt_vn1, wk.hpg, wk.divd2, m.vn, SH(8));
  const T* vn_new = kMixed<T> ? (const T*)m.vn : (const T*)st.vn;
  ICON_LAUNCH(nm_div, blocks_by_shape(SH(6), g.nc, nlev, TH(6)), TH(6), s, (sn_cell_div<T, kTerr>), g, v, vn_new,
              wk.divd, nullptr, nullptr, ex_ref_c, SH(6));
  launch_fluxdiv<T, kTerr>(en, x, vn_new, nm_flx, s);
  if constexpr (kTerr)
    launch_column_terrain<T>(en, 1, st, wk.ddt_w0, wk.ddt_w1, tr.wcc1, s);
  else
    launch_column<T>(en, 1, st, wk.ddt_w0, wk.ddt_w1, s);
}

template <class T>
void launch_substep(const Engine& en, const Ctx<T>& x, const StateView& st, cudaStream_t s) {
  if (en.terrain)
    substep_impl<T, true>(en, x, st, s);
  else
    substep_impl<T, false>(en, x, st, s);
}

template <class T>
void launch_diffusion(const Engine& en, const Ctx<T>& x, const StateView& st, cudaStream_t s) {
  const int* threads = en.threads;
  const GridT<T>& g = x.g;
  const VertT<T>& v = x.v;
  const WorkT<T>& wk = x.w;
  const Mirrors& m = en.m;
  const int nlev = v.nlev, nlevp = nlev + 1;
  const T *s_vn, *s_w, *s_th;
  if constexpr (kMixed<T>) {
    s_vn = m.vn, s_w = m.w, s_th = m.th;
  } else {
    s_vn = st.vn, s_w = st.w, s_th = st.theta_v;
  }
  const long long n1 = (long long)g.nc * nlev + (long long)g.nv * nlev;
  ICON_LAUNCH(kname<T>("diff_div_curl_uv", "diff_div_curl_uv_f32"), blocks_for(n1, TH(9)), TH(9), s,
              diff_div_curl_uv<T>, g, v, s_vn, wk.div_vn, wk.zeta, wk.uv3);
  ICON_LAUNCH(kname<T>("diff_edge_smag", "diff_edge_smag_f32"), blocks_for((long long)g.ne * nlev, TH(10)),
              TH(10), s, diff_edge_smag<T>, g, v, wk.div_vn, wk.zeta, wk.uv3, wk.nu, wk.lap_vn);
  if (x.s.tenh_levels > 0 && x.s.hdiff_temp)
    ICON_LAUNCH(kname<T>("diff_tenh_excess", "diff_tenh_excess_f32"),
                blocks_for((long long)g.nc * x.s.tenh_levels, kThreads), kThreads, s, diff_tenh_excess<T>, g, v, x.s,
                s_th, wk.tenh_ex);
  const long long n3 = (long long)g.nc * nlevp + (long long)g.nv * nlev;
  ICON_LAUNCH(kname<T>("diff_second", "diff_second_f32"), blocks_for(n3, TH(11)), TH(11), s, diff_second<T>, g, v,
              x.s, wk.lap_vn, wk.nu, s_w, s_th, wk.div_l, wk.lap_w, wk.dtheta, wk.curl_l, wk.tenh_ex);
  ICON_LAUNCH(kname<T>("diff_edge_update", "diff_edge_update_f32"), blocks_for((long long)g.ne * nlev, TH(12)),
              TH(12), s, diff_edge_update<T>, g, v, x.s, st.vn, wk.nu, wk.lap_vn, wk.div_l, wk.curl_l, m.vn);
  ICON_LAUNCH(kname<T>("diff_cell_update", "diff_cell_update_f32"), blocks_for((long long)g.nc * nlevp, TH(13)),
              TH(13), s, diff_cell_update<T>, g, v, x.s, en.v.theta_ref, en.v.exner_ref, en.sc.rd_o_cvd, st,
              wk.lap_w, wk.dtheta, m);
}

namespace {
__global__ void fill_kernel(double* p, size_t n, double v) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
}  // namespace

cudaError_t init_va_fused(const VaPatchT& pt) {
  const size_t bytes = va_fused_smem_floats(pt.max_e0, pt.max_e1, pt.max_c3, pt.max_c0, pt.max_v3, pt.max_e4) * sizeof(float);
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(va_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_fill(double* p, size_t n, double v, cudaStream_t s) {
  fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
}

const char* const kStencilNames[kNumStencils] = {
    "va_edge_pre", "va_cell_vert", "va_edge_tend", "va_cell_w", "sn_cell_grad", "sn_edge_pred", "sn_cell_div",
    "sn_cell_fluxdiv", "sn_edge_corr", "diff_div_curl_uv", "diff_edge_smag", "diff_second", "diff_edge_update",
    "diff_cell_update", "va_concorr", "sn_edge_flux"};

void launch_refresh_mirrors(const Engine& en, const StateView& st, cudaStream_t s) {
  const int nlev = en.v.nlev;
  const long long n = (long long)en.g64.ne * nlev + (long long)en.g64.nc * (nlev + 1);
  ICON_LAUNCH("mx_refresh", blocks_for(n, kThreads), kThreads, s, mx_refresh, en.g64.ne, en.g64.nc, nlev,
              en.v.exner_ref, en.v.theta_ref, en.rho_ref64, st, en.m);
}

template void launch_velocity_tendencies<double>(const Ctx<double>&, const double*, const double*, double*, double*,
                                                 const double*, double*, cudaStream_t, const int*, double*,
                                                 const int*);
template void launch_substep<double>(const Engine&, const Ctx<double>&, const StateView&, cudaStream_t);
template void launch_substep<float>(const Engine&, const Ctx<float>&, const StateView&, cudaStream_t);
template void launch_diffusion<double>(const Engine&, const Ctx<double>&, const StateView&, cudaStream_t);
template void launch_diffusion<float>(const Engine&, const Ctx<float>&, const StateView&, cudaStream_t);

}  // namespace icon
