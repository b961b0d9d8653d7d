// MLP building blocks of the learned corrector (internal).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace icon {

// C[M x N] = A[M x K] B[N x K]^T on the tensor cores (tcgen05): bf16 operands,
// K-major, K a multiple of 64, lda/ldb multiples of 8 (>= K), ldc >= N, 16-byte
// aligned operand bases; epilogue: + bias, then either fp32 out or GELU ->
// bf16 out (and the fp32 pre-activation into zpre if given).  Returns an ICON_*
// code (shape and alignment are checked before the launch).
int mlp_gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
              const float* bias, bool gelu_act, float* out_f32, __nv_bfloat16* out_bf16, float* zpre, int ldc,
              cudaStream_t s);
void mlp_transpose(int rows, int cols, const __nv_bfloat16* in, int ldi, __nv_bfloat16* out, int ldo,
                   cudaStream_t s);
void mlp_gelu_backward(int rows, int cols, const float* dh, int ldd, const float* z, int ldz, float* dz32,
                       __nv_bfloat16* dz16, int ldo, cudaStream_t s);
void mlp_to_bf16(int rows, int cols, const float* in, int ldi, __nv_bfloat16* out, int ldo, cudaStream_t s);
void mlp_bias_grad(int rows, int cols, const float* dz, int ldd, float* db, cudaStream_t s);
void mlp_adam(int n_out, int n_in, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
              float eps, float c1, float c2, __nv_bfloat16* wt16, int ldt, __nv_bfloat16* w16, int ldw,
              cudaStream_t s);
void mlp_adam_bias(int n, float* b, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                   float c1, float c2, cudaStream_t s);
// loss = sum (y - t)^2 / (B n_out) (per-row partial sums into rowloss[B]);
// dy = 2 (y - t) / (B n_out)
void mlp_mse(int B, int n_out, const float* y, int ldy, const float* t, int ldt, float* dy, int lddy, double* rowloss,
             cudaStream_t s);

// Device address of the tensor-core GEMM's error word (nonzero once a GEMM gave
// up a bounded wait; sticky).
const int* mlp_tc_error_flag();

// Forward pass of normalised BF16 input rows x16 [B][ldx] (DEVICE; ldx >=
// mlp_input_ld(m), pads zero) without synchronising; B <= max_batch.  *y points
// at the network's own output rows [B][*ldy], valid until its next call.
int mlp_forward_rows(icon_mlp_t* m, const __nv_bfloat16* x16, int ldx, int B, const float** y, int* ldy,
                     cudaStream_t s);
int mlp_input_ld(const icon_mlp_t* m);
int mlp_dims(const icon_mlp_t* m, int* n_in, int* n_out, int* max_batch);
// normalisation statistics (DEVICE, FP32): x_mean and 1/x_std [n_in], y_mean and
// y_std [n_out]; null if unset
void mlp_norm(const icon_mlp_t* m, const float** xm, const float** xis, const float** ym, const float** ys);
// Training data (mlp_data.cu): FP64 column statistics of [rows][n] with the
// group floor (scratch of mlp_stats_scratch_doubles doubles), normalised rows,
// and the random batch of a training step.
size_t mlp_stats_scratch_doubles(int64_t rows, int n);
void mlp_column_stats(const float* x, int64_t rows, int n, const int* groups_dev, int n_groups, double rel_floor,
                      double* scratch, float* mean32, float* sd32, cudaStream_t s);
void mlp_normalise_rows(const float* x, int64_t rows, int n, const float* mean, const float* sd, float* xn,
                        cudaStream_t s);
void mlp_gather_batch(const float* x, int nx, const float* y, int ny, int64_t rows, int batch, uint64_t seed,
                      int64_t step, float* bx, float* by, cudaStream_t s);

}  // namespace icon
