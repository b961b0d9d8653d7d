// Training data of the learned corrector on the GPU (row A13): per-feature
// normalisation statistics of the training rows, their normalised copies, and
// the random row batches of each training step.
//
// Statistics: the mean and the sample standard deviation (divisor rows - 1)
// of every column of a row-major [rows][n] FP32 matrix, accumulated in FP64 in
// two passes (mean, then squared deviations) over fixed row blocks whose
// partial sums are added in a fixed order, so the result is reproducible.  A
// standard deviation below rel_floor times the largest of its feature group
// (consecutive features of one physical field) is raised to that floor, so
// near-constant features are not amplified.
//
// Batches: row i of the batch of training step `step` is row
// splitmix64(seed + 2^32 step + i) mod rows (SplitMix64, Steele, Lea and Flood,
// OOPSLA 2014: a counter-based generator, so no state is kept and a step's
// batch does not depend on the steps before it).
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp.h"

namespace icon {
namespace {

constexpr int kFeat = 32;   // features per block (one warp's lanes)
constexpr int kRowsPerBlock = 2048;

// partial[b][j] = sum over the rows of block b of (x[r][j] - shift[j]) ^ power
__global__ void column_partials(const float* __restrict__ x, int64_t rows, int n, const double* __restrict__ shift,
                                int power, double* __restrict__ partial) {
  const int j = blockIdx.x * kFeat + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * kRowsPerBlock;
  const int64_t r1 = r0 + kRowsPerBlock < rows ? r0 + kRowsPerBlock : rows;
  __shared__ double acc[8][kFeat];
  double s = 0.0;
  if (j < n) {
    const double c = shift ? shift[j] : 0.0;
    for (int64_t r = r0 + threadIdx.y; r < r1; r += blockDim.y) {
      const double d = (double)x[r * n + j] - c;
      s += power == 1 ? d : d * d;
    }
  }
  acc[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    double t = 0.0;
    for (int q = 0; q < (int)blockDim.y; ++q) t += acc[q][threadIdx.x];
    partial[(int64_t)blockIdx.y * n + j] = t;
  }
}

// out[j] = sum_b partial[b][j] in order; mode 0: the mean (/ rows), 1: the sample std (sqrt(/ (rows - 1)))
__global__ void column_reduce(const double* __restrict__ partial, int nb, int n, int64_t rows, int mode,
                              double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partial[(int64_t)b * n + j];
  out[j] = mode == 0 ? t / (double)rows : sqrt(t / (double)(rows > 1 ? rows - 1 : 1));
}

// per group [start[g], start[g+1]): std = max(std, max(top rel_floor, 1e-30)); FP32 statistics out
__global__ void group_floor(const double* __restrict__ mean, double* __restrict__ sd, const int* __restrict__ start,
                            int n_groups, int n, double rel_floor, float* __restrict__ mean32,
                            float* __restrict__ sd32) {
  const int g = blockIdx.x;
  if (g >= n_groups) return;
  const int a = start[g], b = g + 1 < n_groups ? start[g + 1] : n;
  __shared__ double top;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = a; j < b; ++j) t = sd[j] > t ? sd[j] : t;
    top = t;
  }
  __syncthreads();
  const double floor_ = top * rel_floor > 1e-30 ? top * rel_floor : 1e-30;
  for (int j = a + threadIdx.x; j < b; j += blockDim.x) {
    const double s = sd[j] > floor_ ? sd[j] : floor_;
    mean32[j] = (float)mean[j];
    sd32[j] = (float)s;
  }
}

// xn[r][j] = (x[r][j] - mean[j]) / sd[j]
__global__ void normalise_rows(const float* __restrict__ x, int64_t rows, int n, const float* __restrict__ mean,
                               const float* __restrict__ sd, float* __restrict__ xn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * n) return;
  const int j = (int)(i % n);
  xn[i] = (x[i] - mean[j]) / sd[j];
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// dst[i][:] = src[row(i)][:] for the batch rows of a training step, x and y alike
__global__ void gather_batch(const float* __restrict__ x, int nx, const float* __restrict__ y, int ny, int64_t rows,
                             int batch, uint64_t seed, int64_t step, float* __restrict__ bx, float* __restrict__ by) {
  const int i = blockIdx.x;
  if (i >= batch) return;
  const uint64_t r = splitmix64(seed + ((uint64_t)step << 32) + (uint64_t)i) % (uint64_t)rows;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) bx[(int64_t)i * nx + j] = x[(int64_t)r * nx + j];
  for (int j = threadIdx.x; j < ny; j += blockDim.x) by[(int64_t)i * ny + j] = y[(int64_t)r * ny + j];
}

}  // namespace

size_t mlp_stats_scratch_doubles(int64_t rows, int n) {
  const int64_t nb = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  return (size_t)(nb * n + 2 * n);
}

void mlp_column_stats(const float* x, int64_t rows, int n, const int* groups_dev, int n_groups, double rel_floor,
                      double* scratch, float* mean32, float* sd32, cudaStream_t s) {
  const int nb = (int)((rows + kRowsPerBlock - 1) / kRowsPerBlock);
  double* partial = scratch;
  double* mean = scratch + (size_t)nb * n;
  double* sd = mean + n;
  const dim3 grid((n + kFeat - 1) / kFeat, nb), block(kFeat, 8);
  column_partials<<<grid, block, 0, s>>>(x, rows, n, nullptr, 1, partial);
  column_reduce<<<(n + 127) / 128, 128, 0, s>>>(partial, nb, n, rows, 0, mean);
  column_partials<<<grid, block, 0, s>>>(x, rows, n, mean, 2, partial);
  column_reduce<<<(n + 127) / 128, 128, 0, s>>>(partial, nb, n, rows, 1, sd);
  group_floor<<<n_groups, 128, 0, s>>>(mean, sd, groups_dev, n_groups, n, rel_floor, mean32, sd32);
}

void mlp_normalise_rows(const float* x, int64_t rows, int n, const float* mean, const float* sd, float* xn,
                        cudaStream_t s) {
  const int64_t total = rows * n;
  normalise_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, rows, n, mean, sd, xn);
}

void mlp_gather_batch(const float* x, int nx, const float* y, int ny, int64_t rows, int batch, uint64_t seed,
                      int64_t step, float* bx, float* by, cudaStream_t s) {
  gather_batch<<<batch, 128, 0, s>>>(x, nx, y, ny, rows, batch, seed, step, bx, by);
}

}  // namespace icon
