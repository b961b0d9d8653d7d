// Learned corrector (row A13): features of a state for the column and edge
// networks, and the application of their increments to the state.
//
// Column features (5 nlev per cell): w at full levels, exner - exner_ref,
// theta_v - theta_ref, and the cell velocity's east and north components
// (Perot reconstruction).  Edge features (11 nlev per edge): the column
// features of e2c[0] and e2c[1], then vn.  Column outputs (3 nlev - 1):
// increments of w at the interior half levels, of exner and of theta_v; edge
// outputs (nlev): increments of vn.  rho is never changed (mass stays exact).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "kernels.h"

namespace icon {
namespace {

constexpr int kT = 256;

// FP64 -> FP32 by truncation to 24 significant bits with integer operations
// (the features end up in BF16; this keeps them off the FP64 pipe)
__device__ __forceinline__ float f32(double x) { return to_df(x).hi; }

template <class O>
__device__ __forceinline__ O feature_out(float f, const float* mean, const float* istd, int j);
template <>
__device__ __forceinline__ float feature_out<float>(float f, const float* mean, const float* istd, int j) {
  return mean ? (f - mean[j]) * istd[j] : f;
}
template <>
__device__ __forceinline__ __nv_bfloat16 feature_out<__nv_bfloat16>(float f, const float* mean, const float* istd,
                                                                     int j) {
  return __float2bfloat16((f - mean[j]) * istd[j]);
}

// Column features, one thread per (cell, level): raw FP32 rows [nc][5 nlev]
// into raw (if given), and rows [nc][ldx] of type O into x (normalised with
// mean/istd when given; O = BF16 requires them).  The reference profiles are
// per level ([nlev], ref_stride 0) or, over terrain, per column ([nc*nlev],
// ref_stride nlev).
template <class O>
__global__ void col_features(int nc, int nlev, const int* __restrict__ c2e, const float* __restrict__ uv_c,
                             const double* __restrict__ exner_ref, const double* __restrict__ theta_ref,
                             int ref_stride, StateView st, float* __restrict__ raw, O* __restrict__ x, int ldx,
                             const float* __restrict__ mean, const float* __restrict__ istd) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nc * nlev) return;
  const unsigned ui = (unsigned)i;  // < 2^32 (checked by the callers)
  const int c = (int)(ui / (unsigned)nlev), k = (int)(ui - (unsigned)c * (unsigned)nlev);
  const size_t ic = (size_t)c * nlev + k;
  const double* wc = st.w + (size_t)c * (nlev + 1);
  float f[5];
  f[0] = 0.5f * (f32(wc[k]) + f32(wc[k + 1]));
  const size_t ir = (size_t)c * ref_stride + k;
  f[1] = f32(st.exner[ic] - exner_ref[ir]);
  f[2] = f32(st.theta_v[ic] - theta_ref[ir]);
  const int* ce = c2e + 3 * (size_t)c;
  const float* w = uv_c + 6 * (size_t)c;
  float u = 0.f, v = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float vn = f32(st.vn[(size_t)ce[j] * nlev + k]);
    u += w[2 * j] * vn;
    v += w[2 * j + 1] * vn;
  }
  f[3] = u;
  f[4] = v;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int j = q * nlev + k;
    if (raw) raw[(size_t)c * 5 * nlev + j] = f[q];
    if (x) x[(size_t)c * ldx + j] = feature_out<O>(f[q], mean, istd, j);
  }
}

// Edge features, one thread per (edge, level): the raw column features of
// e2c[0] and e2c[1], then vn, into rows [ne][ldx] of type O.
template <class O>
__global__ void edge_features(int ne, int nlev, const int* __restrict__ e2c, const float* __restrict__ colx,
                              const double* __restrict__ vn, O* __restrict__ x, int ldx,
                              const float* __restrict__ mean, const float* __restrict__ istd) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)ne * nlev) return;
  const unsigned ui = (unsigned)i;  // < 2^32 (checked by the callers)
  const int e = (int)(ui / (unsigned)nlev), k = (int)(ui - (unsigned)e * (unsigned)nlev);
  O* xe = x + (size_t)e * ldx;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const float* cx = colx + (size_t)e2c[2 * e + side] * 5 * nlev;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int j = side * 5 * nlev + q * nlev + k;
      xe[j] = feature_out<O>(cx[q * nlev + k], mean, istd, j);
    }
  }
  const int j = 10 * nlev + k;
  xe[j] = feature_out<O>(f32(vn[(size_t)e * nlev + k]), mean, istd, j);
}

// Sum of a value over the block (kT threads) in FP32, by warp shuffles; the
// result in thread 0.  NaN propagates.
__device__ __forceinline__ float block_sum(float s) {
  __shared__ float red[kT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < kT / 32; ++w) t += red[w];
  return t;
}

__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}

// column increments of rows [row0, row0 + rows): y [rows][ldy] normalised ->
// state (FP64 updates); per-block partial sums of y^2 for the correction norm.
// A non-finite new value (or rho) turns the partial into NaN, so the norm test
// also rejects a state that has blown up.
__global__ void apply_col(int row0, int rows, int nlev, const float* __restrict__ y, int ldy,
                          const float* __restrict__ mean, const float* __restrict__ stdv, StateView st,
                          float* __restrict__ partial) {
  const int no = 3 * nlev - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float s = 0.f;
  if (i < (size_t)rows * no) {
    const unsigned ui = (unsigned)i;  // < 2^32 (checked by the callers)
    const int r = (int)(ui / (unsigned)no), j = (int)(ui - (unsigned)r * (unsigned)no);
    const size_t c = (size_t)row0 + r;
    const float yn = y[(size_t)r * ldy + j];
    s = yn * yn;
    const double d = f2d_exact(fmaf(yn, stdv[j], mean[j]));
    double* p;
    if (j < nlev - 1) {
      p = st.w + c * (nlev + 1) + j + 1;
    } else if (j < 2 * nlev - 1) {
      const size_t ic = c * nlev + (j - (nlev - 1));
      p = st.exner + ic;
      if (!finite_bits(st.rho[ic])) s = __int_as_float(0x7fc00000);
    } else {
      p = st.theta_v + c * nlev + (j - (2 * nlev - 1));
    }
    const double v = *p + d;
    *p = v;
    if (!finite_bits(v)) s = __int_as_float(0x7fc00000);
  }
  const float t = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void apply_edge(int row0, int rows, int nlev, const float* __restrict__ y, int ldy,
                           const float* __restrict__ mean, const float* __restrict__ stdv, double* __restrict__ vn,
                           float* __restrict__ partial) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float s = 0.f;
  if (i < (size_t)rows * nlev) {
    const unsigned ui = (unsigned)i;  // < 2^32 (checked by the callers)
    const int r = (int)(ui / (unsigned)nlev), k = (int)(ui - (unsigned)r * (unsigned)nlev);
    const float yn = y[(size_t)r * ldy + k];
    s = yn * yn;
    double* p = vn + ((size_t)row0 + r) * nlev + k;
    const double v = *p + f2d_exact(fmaf(yn, stdv[k], mean[k]));
    *p = v;
    if (!finite_bits(v)) s = __int_as_float(0x7fc00000);
  }
  const float t = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Two-stage fixed-order sums: out[0] = sum of partial[0, n0), out[1] = sum of
// partial[n0, n0 + n1).  Stage 1: kSeg blocks per part each sum one contiguous
// segment into stage[]; stage 2: one block adds the segments in order.
constexpr int kSeg = 64;
__global__ void reduce_stage1(const float* __restrict__ partial, int n0, int n1, double* __restrict__ stage) {
  __shared__ double red[kT];
  const int part = blockIdx.x / kSeg, seg = blockIdx.x - part * kSeg;
  const float* p = partial + (part ? n0 : 0);
  const int n = part ? n1 : n0;
  const int len = (n + kSeg - 1) / kSeg, a = seg * len, b = min(n, a + len);
  double s = 0.0;
  for (int i = a + threadIdx.x; i < b; i += kT) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = kT / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) stage[blockIdx.x] = red[0];
}
__global__ void reduce_stage2(const double* __restrict__ stage, double* __restrict__ out) {
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int i = 0; i < kSeg; ++i) s += stage[threadIdx.x * kSeg + i];
    out[threadIdx.x] = s;
  }
}

// targets: plain - reduced; column [nc][3 nlev - 1] (interior w, exner, theta_v), edge [ne][nlev]
__global__ void col_targets(int nc, int nlev, StateView a, StateView b, float* __restrict__ y) {
  const int no = 3 * nlev - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nc * no) return;
  const unsigned ui = (unsigned)i;  // < 2^32 (checked by the callers)
  const int c = (int)(ui / (unsigned)no), j = (int)(ui - (unsigned)c * (unsigned)no);
  double d;
  if (j < nlev - 1) {
    const size_t ih = (size_t)c * (nlev + 1) + j + 1;
    d = b.w[ih] - a.w[ih];
  } else if (j < 2 * nlev - 1) {
    const size_t ic = (size_t)c * nlev + (j - (nlev - 1));
    d = b.exner[ic] - a.exner[ic];
  } else {
    const size_t ic = (size_t)c * nlev + (j - (2 * nlev - 1));
    d = b.theta_v[ic] - a.theta_v[ic];
  }
  y[i] = (float)d;
}

__global__ void edge_targets(size_t n, const double* __restrict__ a, const double* __restrict__ b,
                             float* __restrict__ y) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)(b[i] - a[i]);
}

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

void launch_col_features(const Engine& en, const StateView& st, float* raw, float* x, int ldx, const float* mean,
                         const float* istd, cudaStream_t s) {
  const int nc = en.g64.nc, nlev = en.v.nlev;
  const bool tr = en.terrain;
  ICON_LAUNCH("lc_col_features", cdiv((size_t)nc * nlev, kT), kT, s, col_features<float>, nc, nlev, en.g64.c2e,
              en.g64.uv_c, tr ? en.v.exner_ref_c : en.v.exner_ref, tr ? en.v.theta_ref_c : en.v.theta_ref,
              tr ? nlev : 0, st, raw, x, ldx, mean, istd);
}

void launch_col_inputs(const Engine& en, const StateView& st, float* raw, __nv_bfloat16* x, int ldx,
                       const float* mean, const float* istd, cudaStream_t s) {
  const int nc = en.g64.nc, nlev = en.v.nlev;
  const bool tr = en.terrain;
  ICON_LAUNCH("lc_col_inputs", cdiv((size_t)nc * nlev, kT), kT, s, col_features<__nv_bfloat16>, nc, nlev,
              en.g64.c2e, en.g64.uv_c, tr ? en.v.exner_ref_c : en.v.exner_ref, tr ? en.v.theta_ref_c : en.v.theta_ref,
              tr ? nlev : 0, st, raw, x, ldx, mean, istd);
}

void launch_edge_features(const Engine& en, const float* colx, const double* vn, float* x, int ldx,
                          const float* mean, const float* istd, cudaStream_t s) {
  const int ne = en.g64.ne, nlev = en.v.nlev;
  ICON_LAUNCH("lc_edge_features", cdiv((size_t)ne * nlev, kT), kT, s, edge_features<float>, ne, nlev, en.g64.e2c,
              colx, vn, x, ldx, mean, istd);
}

void launch_edge_inputs(const Engine& en, const float* colx, const double* vn, __nv_bfloat16* x, int ldx,
                        const float* mean, const float* istd, cudaStream_t s) {
  const int ne = en.g64.ne, nlev = en.v.nlev;
  ICON_LAUNCH("lc_edge_inputs", cdiv((size_t)ne * nlev, kT), kT, s, edge_features<__nv_bfloat16>, ne, nlev,
              en.g64.e2c, colx, vn, x, ldx, mean, istd);
}

int apply_partials(size_t n) { return (int)cdiv(n, kT); }

void launch_apply_col(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                      const float* stdv, const StateView& st, float* partial, cudaStream_t s) {
  const int nlev = en.v.nlev;
  ICON_LAUNCH("lc_apply_col", cdiv((size_t)rows * (3 * nlev - 1), kT), kT, s, apply_col, row0, rows, nlev, y, ldy,
              mean, stdv, st, partial);
}

void launch_apply_edge(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                       const float* stdv, double* vn, float* partial, cudaStream_t s) {
  const int nlev = en.v.nlev;
  ICON_LAUNCH("lc_apply_edge", cdiv((size_t)rows * nlev, kT), kT, s, apply_edge, row0, rows, nlev, y, ldy, mean,
              stdv, vn, partial);
}

int reduce_stage_doubles() { return 2 * kSeg; }

void launch_reduce_status(const float* partial, int n0, int n1, double* stage, double* out, cudaStream_t s) {
  ICON_LAUNCH("lc_reduce_status", 2 * kSeg, kT, s, reduce_stage1, partial, n0, n1, stage);
  ICON_LAUNCH("lc_reduce_status2", 1, 32, s, reduce_stage2, stage, out);
}

void launch_targets(const Engine& en, const StateView& reduced, const StateView& plain, float* col_y, float* edge_y,
                    cudaStream_t s) {
  const int nc = en.g64.nc, ne = en.g64.ne, nlev = en.v.nlev;
  ICON_LAUNCH("lc_col_targets", cdiv((size_t)nc * (3 * nlev - 1), kT), kT, s, col_targets, nc, nlev, reduced, plain,
              col_y);
  const size_t n = (size_t)ne * nlev;
  ICON_LAUNCH("lc_edge_targets", cdiv(n, kT), kT, s, edge_targets, n, reduced.vn, plain.vn, edge_y);
}

}  // namespace icon
