// Learned corrector (row A13): a 3-layer MLP, x -> GELU(x W1 + b1) -> GELU(. W2 + b2)
// -> . W3 + b3, with BF16 weights and activations and FP32 accumulation on the
// tensor cores, plus its backward pass and an Adam update for training on the
// GPU.  GELU is the erf form, 0.5 x (1 + erf(x / sqrt(2))).
//
// Every GEMM is C[M x N] = A[M x K] * B[N x K]^T with both operands K-major
// ("NT"), the layout the warp-level BF16 MMA consumes directly.  Leading
// dimensions are padded to multiples of 64 and the pads hold zeros, so K
// needs no tail handling; ragged M and N are guarded.  The backward GEMMs
// reuse the same kernel on transposed copies (dW^T = dZ^T H, dH = dZ W).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp.h"

namespace icon {
namespace {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int kGemmThreads = 256;  // 8 warps: 2 (M) x 4 (N), warp tile 64 x 32
constexpr int SROW = BK + 8;       // padded shared row (bf16 elements): conflict-free fragment reads

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = pred ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  // d/dx [x Phi(x)] = Phi(x) + x phi(x)
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.3989422804014327f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// Epilogue modes: 0 = fp32 out (+bias if given); 1 = bias + GELU -> bf16 out,
// fp32 pre-activation stored if zpre != null.
struct Epi {
  int mode;
  const float* bias;  // [N] or null
  float* out_f32;     // mode 0
  __nv_bfloat16* out_bf16;  // mode 1
  float* zpre;        // mode 1, optional
  int ldc;
};

__global__ void __launch_bounds__(kGemmThreads) gemm_nt(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                        int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                        Epi ep) {
  __shared__ __align__(16) __nv_bfloat16 As[2][BM * SROW];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][BN * SROW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile origin: (wm*64, wn*32)
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  // each thread copies 2 x 16 bytes of A and 2 x 16 bytes of B per k-tile
  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int idx = tid + r * kGemmThreads;  // 0..511: 128 rows x 4 chunks of 8 bf16
      const int row = idx >> 2, ch = idx & 3;
      const int gm = m0 + row, gn = n0 + row;
      cp_async16(&As[buf][row * SROW + ch * 8], A + (size_t)(gm < M ? gm : 0) * lda + k0 + ch * 8, gm < M);
      cp_async16(&Bs[buf][row * SROW + ch * 8], B + (size_t)(gn < N ? gn : 0) * ldb + k0 + ch * 8, gn < N);
    }
    cp_async_commit();
  };

  const int nk = K / BK;
  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load(buf ^ 1, (kt + 1) * BK);
      cp_async_wait_1();
    } else {
      cp_async_wait_0();
    }
    __syncthreads();
    const __nv_bfloat16* as = As[buf];
    const __nv_bfloat16* bs = Bs[buf];
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r0 = wm * 64 + i * 16 + g;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&as[r0 * SROW + kk + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&as[(r0 + 8) * SROW + kk + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&as[r0 * SROW + kk + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&as[(r0 + 8) * SROW + kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = wn * 32 + j * 8 + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&bs[c0 * SROW + kk + 2 * t]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&bs[c0 * SROW + kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }

  // epilogue
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * 64 + i * 16 + g + (r >= 2 ? 8 : 0);
        const int col = n0 + wn * 32 + j * 8 + 2 * t + (r & 1);
        if (row >= M || col >= N) continue;
        float v = acc[i][j][r];
        if (ep.bias) v += ep.bias[col];
        const size_t o = (size_t)row * ep.ldc + col;
        if (ep.mode == 0) {
          ep.out_f32[o] = v;
        } else {
          if (ep.zpre) ep.zpre[o] = v;
          ep.out_bf16[o] = __float2bfloat16(gelu(v));
        }
      }
}

// out[c][r] = in[r][c] for r < rows, c < cols (bf16); pads of out left untouched
__global__ void transpose_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ in, int ldi,
                               __nv_bfloat16* __restrict__ out, int ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j;
    if (r < rows && c < cols) tile[j][threadIdx.x] = in[(size_t)r * ldi + c];
  }
  __syncthreads();
  const int rr = r0 + threadIdx.x;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int cc = blockIdx.x * 32 + j;
    if (rr < rows && cc < cols) out[(size_t)cc * ldo + rr] = tile[threadIdx.x][j];
  }
}

// dZ = dH * gelu'(Z) (bf16 out for the next GEMMs, fp32 kept for the bias gradient)
__global__ void gelu_backward(int rows, int cols, const float* __restrict__ dh, int ldd,
                              const float* __restrict__ z, int ldz, float* __restrict__ dz32,
                              __nv_bfloat16* __restrict__ dz16, int ldo) {
  const size_t n = (size_t)rows * cols;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = (int)(i / cols), c = (int)(i - (size_t)r * cols);
  const float v = dh[(size_t)r * ldd + c] * gelu_grad(z[(size_t)r * ldz + c]);
  dz32[(size_t)r * ldo + c] = v;
  dz16[(size_t)r * ldo + c] = __float2bfloat16(v);
}

// fp32 -> bf16 copy with padding (pads written as zero)
__global__ void to_bf16(int rows, int cols, const float* __restrict__ in, int ldi, __nv_bfloat16* __restrict__ out,
                        int ldo) {
  const size_t n = (size_t)rows * ldo;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = (int)(i / ldo), c = (int)(i - (size_t)r * ldo);
  out[i] = __float2bfloat16(c < cols ? in[(size_t)r * ldi + c] : 0.f);
}

// db[c] = sum_r dz[r][c], fixed order per column (one thread per column)
__global__ void bias_grad(int rows, int cols, const float* __restrict__ dz, int ldd, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dz[(size_t)r * ldd + c];
  db[c] = s;
}

// Adam on fp32 master weights; refreshes the bf16 copy W^T [n][k] and W [k][n]
__global__ void adam_update(int n_out, int n_in, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* __restrict__ wt16, int ldt,
                            __nv_bfloat16* __restrict__ w16, int ldw) {
  const size_t n = (size_t)n_out * n_in;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wt16) {
    const int o = (int)(i / n_in), k = (int)(i - (size_t)o * n_in);
    wt16[(size_t)o * ldt + k] = __float2bfloat16(wi);
    w16[(size_t)k * ldw + o] = __float2bfloat16(wi);
  }
}

__global__ void adam_update_bias(int n, float* __restrict__ b, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  b[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

void mlp_gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
              const float* bias, bool gelu_act, float* out_f32, __nv_bfloat16* out_bf16, float* zpre, int ldc,
              cudaStream_t s) {
  Epi ep{gelu_act ? 1 : 0, bias, out_f32, out_bf16, zpre, ldc};
  dim3 grid(cdiv(N, BN), cdiv(M, BM));
  ICON_LAUNCH("mlp_gemm", grid, kGemmThreads, s, gemm_nt, M, N, K, A, lda, B, ldb, ep);
}

void mlp_transpose(int rows, int cols, const __nv_bfloat16* in, int ldi, __nv_bfloat16* out, int ldo,
                   cudaStream_t s) {
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  ICON_LAUNCH("mlp_transpose", grid, dim3(32, 8), s, transpose_bf16, rows, cols, in, ldi, out, ldo);
}

void mlp_gelu_backward(int rows, int cols, const float* dh, int ldd, const float* z, int ldz, float* dz32,
                       __nv_bfloat16* dz16, int ldo, cudaStream_t s) {
  ICON_LAUNCH("mlp_gelu_backward", cdiv((size_t)rows * cols, 256), 256, s, gelu_backward, rows, cols, dh, ldd, z,
              ldz, dz32, dz16, ldo);
}

void mlp_to_bf16(int rows, int cols, const float* in, int ldi, __nv_bfloat16* out, int ldo, cudaStream_t s) {
  ICON_LAUNCH("mlp_to_bf16", cdiv((size_t)rows * ldo, 256), 256, s, to_bf16, rows, cols, in, ldi, out, ldo);
}

void mlp_bias_grad(int rows, int cols, const float* dz, int ldd, float* db, cudaStream_t s) {
  ICON_LAUNCH("mlp_bias_grad", cdiv(cols, 128), 128, s, bias_grad, rows, cols, dz, ldd, db);
}

void mlp_adam(int n_out, int n_in, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
              float eps, float c1, float c2, __nv_bfloat16* wt16, int ldt, __nv_bfloat16* w16, int ldw,
              cudaStream_t s) {
  ICON_LAUNCH("mlp_adam", cdiv((size_t)n_out * n_in, 256), 256, s, adam_update, n_out, n_in, w, g, m, v, lr, b1, b2,
              eps, c1, c2, wt16, ldt, w16, ldw);
}

void mlp_adam_bias(int n, float* b, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                   float c1, float c2, cudaStream_t s) {
  ICON_LAUNCH("mlp_adam_bias", cdiv(n, 256), 256, s, adam_update_bias, n, b, g, m, v, lr, b1, b2, eps, c1, c2);
}

}  // namespace icon

namespace icon {
namespace {
__global__ void mse_kernel(int B, int n_out, const float* __restrict__ y, int ldy, const float* __restrict__ t,
                           int ldt, float* __restrict__ dy, int lddy, double* __restrict__ rowloss) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const float scale = 2.0f / ((float)B * (float)n_out);
  double s = 0.0;
  for (int c = 0; c < n_out; ++c) {
    const float d = y[(size_t)r * ldy + c] - t[(size_t)r * ldt + c];
    s += (double)d * d;
    dy[(size_t)r * lddy + c] = scale * d;
  }
  rowloss[r] = s;
}
}  // namespace

void mlp_mse(int B, int n_out, const float* y, int ldy, const float* t, int ldt, float* dy, int lddy, double* rowloss,
             cudaStream_t s) {
  ICON_LAUNCH("mlp_mse", (unsigned)((B + 127) / 128), 128, s, mse_kernel, B, n_out, y, ldy, t, ldt, dy, lddy,
              rowloss);
}

}  // namespace icon
