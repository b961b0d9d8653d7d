// Learned corrector (row A13): features of a state for the column and edge
// networks, and the application of their increments to the state.
//
// Column features (5 nlev per cell): w at full levels, exner - exner_ref,
// theta_v - theta_ref, and the cell velocity's east and north components
// (Perot reconstruction).  Edge features (11 nlev per edge): the column
// features of e2c[0] and e2c[1], then vn.  Column outputs (3 nlev - 1):
// increments of w at the interior half levels, of exner and of theta_v; edge
// outputs (nlev): increments of vn.  rho is never changed (mass stays exact).
#include <cuda_runtime.h>

#include "kernels.h"

namespace icon {
namespace {

constexpr int kT = 256;

// raw column features [nc][5 nlev]; one thread per (cell, level)
__global__ void col_features(int nc, int nlev, const int* __restrict__ c2e, const float* __restrict__ uv_c,
                             const double* __restrict__ exner_ref, const double* __restrict__ theta_ref,
                             StateView st, float* __restrict__ x) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nc * nlev) return;
  const int c = (int)(i / nlev), k = (int)(i - (size_t)c * nlev);
  const size_t ic = (size_t)c * nlev + k;
  float* xc = x + (size_t)c * 5 * nlev;
  const double* wc = st.w + (size_t)c * (nlev + 1);
  xc[k] = (float)(0.5 * (wc[k] + wc[k + 1]));
  xc[nlev + k] = (float)(st.exner[ic] - exner_ref[k]);
  xc[2 * nlev + k] = (float)(st.theta_v[ic] - theta_ref[k]);
  const int* ce = c2e + 3 * (size_t)c;
  const float* w = uv_c + 6 * (size_t)c;
  float u = 0.f, v = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float vn = (float)st.vn[(size_t)ce[j] * nlev + k];
    u += w[2 * j] * vn;
    v += w[2 * j + 1] * vn;
  }
  xc[3 * nlev + k] = u;
  xc[4 * nlev + k] = v;
}

// edge features [ne][11 nlev] from raw column features, normalised with (mean, std) if given
__global__ void edge_features(int ne, int nlev, const int* __restrict__ e2c, const float* __restrict__ colx,
                              const double* __restrict__ vn, const float* __restrict__ mean,
                              const float* __restrict__ stdv, float* __restrict__ x) {
  const int nf = 11 * nlev;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)ne * nf) return;
  const int e = (int)(i / nf), j = (int)(i - (size_t)e * nf);
  float f;
  if (j < 10 * nlev) {
    const int side = j < 5 * nlev ? 0 : 1;
    f = colx[(size_t)e2c[2 * e + side] * 5 * nlev + (j - side * 5 * nlev)];
  } else {
    f = (float)vn[(size_t)e * nlev + (j - 10 * nlev)];
  }
  if (mean) f = (f - mean[j]) / stdv[j];
  x[i] = f;
}

// in-place normalisation of rows [n][nf] with per-feature (mean, std)
__global__ void normalise(size_t n, int nf, float* __restrict__ x, const float* __restrict__ mean,
                          const float* __restrict__ stdv) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n * nf) return;
  const int j = (int)(i % nf);
  x[i] = (x[i] - mean[j]) / stdv[j];
}

// column increments of rows [row0, row0 + rows): y [rows][ldy] normalised ->
// state (FP64 updates); per-block partial sums of y^2 for the correction norm.
// A non-finite new value (or rho) turns the partial into NaN, so the norm test
// also rejects a state that has blown up.
__global__ void apply_col(int row0, int rows, int nlev, const float* __restrict__ y, int ldy,
                          const float* __restrict__ mean, const float* __restrict__ stdv, StateView st,
                          double* __restrict__ partial) {
  __shared__ double red[kT];
  const int no = 3 * nlev - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < (size_t)rows * no) {
    const int r = (int)(i / no), j = (int)(i - (size_t)r * no);
    const size_t c = (size_t)row0 + r;
    const float yn = y[(size_t)r * ldy + j];
    s = (double)yn * yn;
    const double d = (double)(yn * stdv[j] + mean[j]);
    double* p;
    if (j < nlev - 1) {
      p = st.w + c * (nlev + 1) + j + 1;
    } else if (j < 2 * nlev - 1) {
      const size_t ic = c * nlev + (j - (nlev - 1));
      p = st.exner + ic;
      if (!isfinite(st.rho[ic])) s = nan("");
    } else {
      p = st.theta_v + c * nlev + (j - (2 * nlev - 1));
    }
    const double v = *p + d;
    *p = v;
    if (!isfinite(v)) s = nan("");
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = kT / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void apply_edge(int row0, int rows, int nlev, const float* __restrict__ y, int ldy,
                           const float* __restrict__ mean, const float* __restrict__ stdv, double* __restrict__ vn,
                           double* __restrict__ partial) {
  __shared__ double red[kT];
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < (size_t)rows * nlev) {
    const int r = (int)(i / nlev), k = (int)(i - (size_t)r * nlev);
    const float yn = y[(size_t)r * ldy + k];
    s = (double)yn * yn;
    double* p = vn + ((size_t)row0 + r) * nlev + k;
    const double v = *p + (double)(yn * stdv[k] + mean[k]);
    *p = v;
    if (!isfinite(v)) s = nan("");
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = kT / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[0] = sum of partial[0, n0), out[1] = sum of partial[n0, n0 + n1); one
// block, fixed summation order
__global__ void reduce_status(const double* __restrict__ partial, int n0, int n1, double* __restrict__ out) {
  __shared__ double red[1024];
  for (int part = 0; part < 2; ++part) {
    const double* p = partial + (part ? n0 : 0);
    const int n = part ? n1 : n0;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 512; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[part] = red[0];
    __syncthreads();
  }
}

// targets: plain - reduced; column [nc][3 nlev - 1] (interior w, exner, theta_v), edge [ne][nlev]
__global__ void col_targets(int nc, int nlev, StateView a, StateView b, float* __restrict__ y) {
  const int no = 3 * nlev - 1;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nc * no) return;
  const int c = (int)(i / no), j = (int)(i - (size_t)c * no);
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

void launch_col_features(const Engine& en, const StateView& st, float* x, cudaStream_t s) {
  const int nc = en.g64.nc, nlev = en.v.nlev;
  ICON_LAUNCH("lc_col_features", cdiv((size_t)nc * nlev, kT), kT, s, col_features, nc, nlev, en.g64.c2e,
              en.g64.uv_c, en.v.exner_ref, en.v.theta_ref, st, x);
}

void launch_edge_features(const Engine& en, const float* colx, const double* vn, const float* mean,
                          const float* stdv, float* x, cudaStream_t s) {
  const int ne = en.g64.ne, nlev = en.v.nlev;
  ICON_LAUNCH("lc_edge_features", cdiv((size_t)ne * 11 * nlev, kT), kT, s, edge_features, ne, nlev, en.g64.e2c, colx,
              vn, mean, stdv, x);
}

void launch_normalise(size_t n, int nf, float* x, const float* mean, const float* stdv, cudaStream_t s) {
  ICON_LAUNCH("lc_normalise", cdiv(n * nf, kT), kT, s, normalise, n, nf, x, mean, stdv);
}

int apply_partials(size_t n) { return (int)cdiv(n, kT); }

void launch_apply_col(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                      const float* stdv, const StateView& st, double* partial, cudaStream_t s) {
  const int nlev = en.v.nlev;
  ICON_LAUNCH("lc_apply_col", cdiv((size_t)rows * (3 * nlev - 1), kT), kT, s, apply_col, row0, rows, nlev, y, ldy,
              mean, stdv, st, partial);
}

void launch_apply_edge(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                       const float* stdv, double* vn, double* partial, cudaStream_t s) {
  const int nlev = en.v.nlev;
  ICON_LAUNCH("lc_apply_edge", cdiv((size_t)rows * nlev, kT), kT, s, apply_edge, row0, rows, nlev, y, ldy, mean,
              stdv, vn, partial);
}

void launch_reduce_status(const double* partial, int n0, int n1, double* out, cudaStream_t s) {
  ICON_LAUNCH("lc_reduce_status", 1, 1024, s, reduce_status, partial, n0, n1, out);
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
