// C-ABI of the learned corrector's MLP (row A13): parameters, forward,
// backward, Adam and a fused training step, all on the GPU.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mlp.h"

using namespace icon;

struct icon_mlp {
  int dims[4];   // n_in, n_hidden, n_hidden, n_out
  int lds[4];    // padded to multiples of 64
  int max_batch, ld_b;
  int adam_t = 0;
  std::vector<void*> allocs;
  float *w[3], *b[3], *gw[3], *gb[3], *mw[3], *vw[3], *mb[3], *vb[3];
  __nv_bfloat16 *wt16[3], *w16[3];
  // activations (max_batch rows)
  __nv_bfloat16 *x16, *h16[2];
  float *z[2], *y;
  // backward work
  float *dy, *dh, *dz32;
  __nv_bfloat16 *dz16, *dzT, *hT;
  double* rowloss;
  float *x_mean = nullptr, *x_istd = nullptr, *y_mean = nullptr, *y_std = nullptr;  // normalisation
  float *x_std = nullptr;                 // the input standard deviations themselves (icon_mlp_get_normalization)
  float *bx = nullptr, *by = nullptr;     // a sampled training batch [max_batch][n_in], [max_batch][n_out]
};

namespace {

int pad64(int x) { return (x + 63) / 64 * 64; }

int fail_m(int code, const std::string& m) { return report_error(code, m); }

template <class T>
T* alloc(icon_mlp* m, size_t n, cudaError_t& st) {
  if (st != cudaSuccess) return nullptr;
  void* p = nullptr;
  st = cudaMalloc(&p, n * sizeof(T));
  if (st == cudaSuccess) {
    st = cudaMemset(p, 0, n * sizeof(T));
    m->allocs.push_back(p);
  }
  return static_cast<T*>(p);
}

int layer_in(const icon_mlp* m, int l) { return m->dims[l]; }
int layer_out(const icon_mlp* m, int l) { return m->dims[l + 1]; }

// device buffers of the normalisation statistics (allocated on first use)
cudaError_t ensure_norm(icon_mlp* m) {
  cudaError_t st = cudaSuccess;
  if (!m->x_mean) {
    m->x_mean = alloc<float>(m, m->dims[0], st);
    m->x_istd = alloc<float>(m, m->dims[0], st);
    m->x_std = alloc<float>(m, m->dims[0], st);
    m->y_mean = alloc<float>(m, m->dims[3], st);
    m->y_std = alloc<float>(m, m->dims[3], st);
  }
  return st;
}

__global__ void reciprocal_kernel(const float* __restrict__ x, float* __restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = 1.0f / x[i];
}

int64_t param_count(const icon_mlp* m) {
  int64_t n = 0;
  for (int l = 0; l < 3; ++l) n += (int64_t)layer_out(m, l) * layer_in(m, l) + layer_out(m, l);
  return n;
}

// The three layers on BF16 input rows x16 [B][ldx] (ldx >= lds[0], pads zero);
// keep_z: store the FP32 pre-activations a following backward needs
int forward_from(icon_mlp* m, const __nv_bfloat16* x16, int ldx, int B, cudaStream_t s, bool keep_z) {
  const __nv_bfloat16* in = x16;
  int ld = ldx;
  for (int l = 0; l < 2; ++l) {
    int rc = mlp_gemm(B, layer_out(m, l), m->lds[l], in, ld, m->wt16[l], m->lds[l], m->b[l], true, nullptr,
                      m->h16[l], keep_z ? m->z[l] : nullptr, m->lds[l + 1], s);
    if (rc != ICON_OK) return rc;
    in = m->h16[l];
    ld = m->lds[l + 1];
  }
  return mlp_gemm(B, layer_out(m, 2), m->lds[2], in, m->lds[2], m->wt16[2], m->lds[2], m->b[2], false, m->y, nullptr,
                  nullptr, m->lds[3], s);
}

// FP32 input rows [B][n_in]: converted into the network's own BF16 buffer first
int forward(icon_mlp* m, const float* x, int B, cudaStream_t s, bool keep_z = true) {
  mlp_to_bf16(B, m->dims[0], x, m->dims[0], m->x16, m->lds[0], s);
  return forward_from(m, m->x16, m->lds[0], B, s, keep_z);
}

// gradients of all parameters for dL/dy in m->dy (fp32 [B][lds[3]]), after
// forward(); B a multiple of 64 (the K extent of the weight-gradient GEMMs)
int backward(icon_mlp* m, int B, cudaStream_t s) {
  // layer 3 (no activation): dz = dy
  const int n3 = layer_out(m, 2);
  mlp_to_bf16(B, n3, m->dy, m->lds[3], m->dz16, m->lds[3], s);
  mlp_bias_grad(B, n3, m->dy, m->lds[3], m->gb[2], s);
  int ldz = m->lds[3];
  for (int l = 2; l >= 0; --l) {
    const int nin = layer_in(m, l), nout = layer_out(m, l);
    const __nv_bfloat16* h = l == 0 ? m->x16 : m->h16[l - 1];
    // dW^T [nout][nin] = dZ^T H over the batch
    mlp_transpose(B, nout, m->dz16, ldz, m->dzT, m->ld_b, s);
    mlp_transpose(B, nin, h, m->lds[l], m->hT, m->ld_b, s);
    int rc = mlp_gemm(nout, nin, B, m->dzT, m->ld_b, m->hT, m->ld_b, nullptr, false, m->gw[l], nullptr, nullptr, nin,
                      s);
    if (rc != ICON_OK) return rc;
    if (l == 0) break;
    // dH [B][nin] = dZ W (W stored [nin][lds[l+1]])
    rc = mlp_gemm(B, nin, m->lds[l + 1], m->dz16, ldz, m->w16[l], m->lds[l + 1], nullptr, false, m->dh, nullptr,
                  nullptr, m->lds[l], s);
    if (rc != ICON_OK) return rc;
    // dZ of the previous layer through its GELU
    mlp_gelu_backward(B, nin, m->dh, m->lds[l], m->z[l - 1], m->lds[l], m->dz32, m->dz16, m->lds[l], s);
    mlp_bias_grad(B, nin, m->dz32, m->lds[l], m->gb[l - 1], s);
    ldz = m->lds[l];
  }
  return ICON_OK;
}

void adam(icon_mlp* m, float lr, float b1, float b2, float eps, cudaStream_t s) {
  m->adam_t += 1;
  const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
  for (int l = 0; l < 3; ++l) {
    const int nin = layer_in(m, l), nout = layer_out(m, l);
    mlp_adam(nout, nin, m->w[l], m->gw[l], m->mw[l], m->vw[l], lr, b1, b2, eps, c1, c2, m->wt16[l], m->lds[l],
             m->w16[l], m->lds[l + 1], s);
    mlp_adam_bias(nout, m->b[l], m->gb[l], m->mb[l], m->vb[l], lr, b1, b2, eps, c1, c2, s);
  }
}

__global__ void refresh_bf16(int n_out, int n_in, const float* __restrict__ w, __nv_bfloat16* __restrict__ wt16,
                             int ldt, __nv_bfloat16* __restrict__ w16, int ldw) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)n_out * n_in) return;
  const int o = (int)(i / n_in), k = (int)(i - (size_t)o * n_in);
  wt16[(size_t)o * ldt + k] = __float2bfloat16(w[i]);
  w16[(size_t)k * ldw + o] = __float2bfloat16(w[i]);
}

// ICON_ERR_CUDA once a tensor-core GEMM has given up a bounded wait (synchronous read)
int tc_status(const char* fn) {
  const int* flag = mlp_tc_error_flag();
  int v = 0;
  if (!flag || cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_m(ICON_ERR_CUDA, std::string(fn) + ": cannot read the GEMM status");
  if (v) return fail_m(ICON_ERR_CUDA, std::string(fn) + ": a tensor-core GEMM timed out waiting for its pipeline");
  return ICON_OK;
}

int check_batch(const icon_mlp* m, int B, const char* fn) {
  if (B < 1 || B > m->max_batch) return fail_m(ICON_ERR_ARG, std::string(fn) + ": batch out of range");
  return ICON_OK;
}

}  // namespace

namespace icon {
int mlp_forward_rows(icon_mlp_t* m, const __nv_bfloat16* x16, int ldx, int B, const float** y, int* ldy,
                     cudaStream_t s) {
  if (B < 1 || B > m->max_batch) return fail_m(ICON_ERR_ARG, "corrector: batch out of range");
  if (ldx < m->lds[0]) return fail_m(ICON_ERR_ARG, "corrector: input rows too short");
  const int rc = forward_from(m, x16, ldx, B, s, false);
  if (rc != ICON_OK) return rc;
  *y = m->y;
  *ldy = m->lds[3];
  return ICON_OK;
}
int mlp_input_ld(const icon_mlp_t* m) { return m->lds[0]; }
int mlp_dims(const icon_mlp_t* m, int* n_in, int* n_out, int* max_batch) {
  *n_in = m->dims[0];
  *n_out = m->dims[3];
  *max_batch = m->max_batch;
  return ICON_OK;
}
void mlp_norm(const icon_mlp_t* m, const float** xm, const float** xis, const float** ym, const float** ys) {
  *xm = m->x_mean;
  *xis = m->x_istd;
  *ym = m->y_mean;
  *ys = m->y_std;
}
}  // namespace icon

extern "C" {

int icon_mlp_set_normalization(icon_mlp_t* m, const float* x_mean, const float* x_std, const float* y_mean,
                               const float* y_std) {
  if (!m || !x_mean || !x_std || !y_mean || !y_std) return fail_m(ICON_ERR_ARG, "icon_mlp_set_normalization: NULL");
  std::vector<float> istd(m->dims[0]);
  for (int j = 0; j < m->dims[0]; ++j) {
    if (!(x_std[j] > 0.0f)) return fail_m(ICON_ERR_ARG, "icon_mlp_set_normalization: x_std must be positive");
    istd[j] = 1.0f / x_std[j];
  }
  cudaError_t st = cudaSuccess;
  st = ensure_norm(m);
  if (st == cudaSuccess) st = cudaMemcpy(m->x_std, x_std, m->dims[0] * 4, cudaMemcpyHostToDevice);
  if (st == cudaSuccess) st = cudaMemcpy(m->x_mean, x_mean, m->dims[0] * 4, cudaMemcpyHostToDevice);
  if (st == cudaSuccess) st = cudaMemcpy(m->x_istd, istd.data(), m->dims[0] * 4, cudaMemcpyHostToDevice);
  if (st == cudaSuccess) st = cudaMemcpy(m->y_mean, y_mean, m->dims[3] * 4, cudaMemcpyHostToDevice);
  if (st == cudaSuccess) st = cudaMemcpy(m->y_std, y_std, m->dims[3] * 4, cudaMemcpyHostToDevice);
  if (st != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_set_normalization: ") + cudaGetErrorString(st));
  return ICON_OK;
}

int icon_mlp_get_normalization(const icon_mlp_t* m, float* x_mean, float* x_std, float* y_mean, float* y_std) {
  if (!m || !x_mean || !x_std || !y_mean || !y_std) return fail_m(ICON_ERR_ARG, "icon_mlp_get_normalization: NULL");
  if (!m->x_mean) return fail_m(ICON_ERR_ARG, "icon_mlp_get_normalization: the network has no statistics");
  cudaError_t st = cudaMemcpy(x_mean, m->x_mean, m->dims[0] * 4, cudaMemcpyDeviceToHost);
  if (st == cudaSuccess) st = cudaMemcpy(x_std, m->x_std, m->dims[0] * 4, cudaMemcpyDeviceToHost);
  if (st == cudaSuccess) st = cudaMemcpy(y_mean, m->y_mean, m->dims[3] * 4, cudaMemcpyDeviceToHost);
  if (st == cudaSuccess) st = cudaMemcpy(y_std, m->y_std, m->dims[3] * 4, cudaMemcpyDeviceToHost);
  if (st != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_get_normalization: ") + cudaGetErrorString(st));
  return ICON_OK;
}

int icon_mlp_fit_normalization(icon_mlp_t* m, const float* x, const float* y, int64_t rows, const int32_t* x_groups,
                               int32_t n_x_groups, const int32_t* y_groups, int32_t n_y_groups, float rel_floor,
                               float* xn, float* yn, void* stream) {
  const char* fn = "icon_mlp_fit_normalization: ";
  if (!m || !x || !y || !xn || !yn || !x_groups || !y_groups) return fail_m(ICON_ERR_ARG, std::string(fn) + "NULL");
  if (rows < 2 || n_x_groups < 1 || n_y_groups < 1 || !(rel_floor >= 0.0f))
    return fail_m(ICON_ERR_ARG, std::string(fn) + "need rows >= 2, groups and rel_floor >= 0");
  const int nx = m->dims[0], ny = m->dims[3];
  for (int k = 0; k < 2; ++k) {
    const int32_t* gr = k ? y_groups : x_groups;
    const int ng = k ? n_y_groups : n_x_groups, n = k ? ny : nx;
    for (int g = 0; g < ng; ++g)
      if (gr[g] < 0 || gr[g] >= n || (g > 0 && gr[g] <= gr[g - 1]) || (g == 0 && gr[0] != 0))
        return fail_m(ICON_ERR_ARG, std::string(fn) + "groups must start at 0 and increase within the features");
  }
  cudaError_t st = ensure_norm(m);
  if (st != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(st));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch of this call only (the training set is sized by the caller)
  const size_t nd = mlp_stats_scratch_doubles(rows, nx > ny ? nx : ny);
  double* scratch = nullptr;
  int* groups = nullptr;
  st = cudaMalloc(&scratch, nd * sizeof(double));
  if (st == cudaSuccess) st = cudaMalloc(&groups, (n_x_groups + n_y_groups) * sizeof(int));
  if (st == cudaSuccess)
    st = cudaMemcpyAsync(groups, x_groups, n_x_groups * sizeof(int), cudaMemcpyHostToDevice, s);
  if (st == cudaSuccess)
    st = cudaMemcpyAsync(groups + n_x_groups, y_groups, n_y_groups * sizeof(int), cudaMemcpyHostToDevice, s);
  if (st == cudaSuccess) {
    mlp_column_stats(x, rows, nx, groups, n_x_groups, rel_floor, scratch, m->x_mean, m->x_std, s);
    mlp_column_stats(y, rows, ny, groups + n_x_groups, n_y_groups, rel_floor, scratch, m->y_mean, m->y_std, s);
    reciprocal_kernel<<<(nx + 127) / 128, 128, 0, s>>>(m->x_std, m->x_istd, nx);
    mlp_normalise_rows(x, rows, nx, m->x_mean, m->x_std, xn, s);
    mlp_normalise_rows(y, rows, ny, m->y_mean, m->y_std, yn, s);
    st = cudaGetLastError();
  }
  // the host arrays and the scratch are released only after the GPU used them
  const cudaError_t sy = cudaStreamSynchronize(s);
  if (st == cudaSuccess) st = sy;
  cudaFree(scratch);
  cudaFree(groups);
  if (st != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(st));
  return ICON_OK;
}

int icon_mlp_train_step_sampled(icon_mlp_t* m, const float* xn, const float* yn, int64_t rows, int32_t batch,
                                uint64_t seed, int64_t step, float lr, double* loss, void* stream) {
  const char* fn = "icon_mlp_train_step_sampled: ";
  if (!m || !xn || !yn) return fail_m(ICON_ERR_ARG, std::string(fn) + "NULL argument");
  if (rows < 1 || batch < 64 || batch % 64 || batch > m->max_batch)
    return fail_m(ICON_ERR_ARG, std::string(fn) + "need rows >= 1 and batch a multiple of 64 up to max_batch");
  cudaError_t st = cudaSuccess;
  if (!m->bx) {
    m->bx = alloc<float>(m, (size_t)m->max_batch * m->dims[0], st);
    m->by = alloc<float>(m, (size_t)m->max_batch * m->dims[3], st);
  }
  if (st != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string(fn) + cudaGetErrorString(st));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_gather_batch(xn, m->dims[0], yn, m->dims[3], rows, batch, seed, step, m->bx, m->by, s);
  return icon_mlp_train_step(m, m->bx, m->by, batch, lr, loss, stream);
}

int icon_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, icon_mlp_t** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 64 || max_batch % 64)
    return fail_m(ICON_ERR_ARG, "icon_mlp_create: bad sizes (max_batch must be a positive multiple of 64)");
  *out = nullptr;
  icon_mlp* m = new (std::nothrow) icon_mlp();
  if (!m) return fail_m(ICON_ERR_ARG, "icon_mlp_create: out of host memory");
  m->dims[0] = n_in;
  m->dims[1] = m->dims[2] = n_hidden;
  m->dims[3] = n_out;
  for (int i = 0; i < 4; ++i) m->lds[i] = pad64(m->dims[i]);
  m->max_batch = max_batch;
  m->ld_b = max_batch;
  cudaError_t st = cudaSuccess;
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)layer_out(m, l) * layer_in(m, l), nb = layer_out(m, l);
    m->w[l] = alloc<float>(m, nw, st);
    m->gw[l] = alloc<float>(m, nw, st);
    m->mw[l] = alloc<float>(m, nw, st);
    m->vw[l] = alloc<float>(m, nw, st);
    m->b[l] = alloc<float>(m, nb, st);
    m->gb[l] = alloc<float>(m, nb, st);
    m->mb[l] = alloc<float>(m, nb, st);
    m->vb[l] = alloc<float>(m, nb, st);
    m->wt16[l] = alloc<__nv_bfloat16>(m, (size_t)layer_out(m, l) * m->lds[l], st);
    m->w16[l] = alloc<__nv_bfloat16>(m, (size_t)layer_in(m, l) * m->lds[l + 1], st);
  }
  const size_t B = max_batch;
  int ldmax = 0;
  for (int i = 0; i < 4; ++i) ldmax = m->lds[i] > ldmax ? m->lds[i] : ldmax;
  m->x16 = alloc<__nv_bfloat16>(m, B * m->lds[0], st);
  for (int l = 0; l < 2; ++l) {
    m->h16[l] = alloc<__nv_bfloat16>(m, B * m->lds[l + 1], st);
    m->z[l] = alloc<float>(m, B * m->lds[l + 1], st);
  }
  m->y = alloc<float>(m, B * m->lds[3], st);
  m->dy = alloc<float>(m, B * m->lds[3], st);
  m->dh = alloc<float>(m, B * ldmax, st);
  m->dz32 = alloc<float>(m, B * ldmax, st);
  m->dz16 = alloc<__nv_bfloat16>(m, B * ldmax, st);
  m->dzT = alloc<__nv_bfloat16>(m, (size_t)ldmax * B, st);
  m->hT = alloc<__nv_bfloat16>(m, (size_t)ldmax * B, st);
  m->rowloss = alloc<double>(m, B, st);
  if (st != cudaSuccess) {
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_create: ") + cudaGetErrorString(st));
  }
  *out = m;
  return ICON_OK;
}

int icon_mlp_destroy(icon_mlp_t* m) {
  if (!m) return ICON_OK;
  cudaDeviceSynchronize();
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return ICON_OK;
}

int64_t icon_mlp_param_count(const icon_mlp_t* m) { return m ? param_count(m) : -1; }

int icon_mlp_set_params(icon_mlp_t* m, const float* host, int64_t n) {
  if (!m || !host || n != param_count(m)) return fail_m(ICON_ERR_ARG, "icon_mlp_set_params: NULL or wrong count");
  int64_t off = 0;
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)layer_out(m, l) * layer_in(m, l), nb = layer_out(m, l);
    if (cudaMemcpy(m->w[l], host + off, nw * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->b[l], host + off + nw, nb * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_m(ICON_ERR_CUDA, "icon_mlp_set_params: copy failed");
    off += nw + nb;
    cudaMemset(m->mw[l], 0, nw * 4);
    cudaMemset(m->vw[l], 0, nw * 4);
    cudaMemset(m->mb[l], 0, nb * 4);
    cudaMemset(m->vb[l], 0, nb * 4);
    refresh_bf16<<<(unsigned)((nw + 255) / 256), 256>>>(layer_out(m, l), layer_in(m, l), m->w[l], m->wt16[l],
                                                         m->lds[l], m->w16[l], m->lds[l + 1]);
  }
  m->adam_t = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_set_params: ") + cudaGetErrorString(e));
  return ICON_OK;
}

static int copy_out(const icon_mlp* m, float* host, int64_t n, bool grads, const char* fn) {
  if (!m || !host || n != param_count(m)) return fail_m(ICON_ERR_ARG, std::string(fn) + ": NULL or wrong count");
  cudaDeviceSynchronize();
  int64_t off = 0;
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)layer_out(m, l) * layer_in(m, l), nb = layer_out(m, l);
    if (cudaMemcpy(host + off, grads ? m->gw[l] : m->w[l], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host + off + nw, grads ? m->gb[l] : m->b[l], nb * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail_m(ICON_ERR_CUDA, std::string(fn) + ": copy failed");
    off += nw + nb;
  }
  return ICON_OK;
}

int icon_mlp_get_params(const icon_mlp_t* m, float* host, int64_t n) {
  return copy_out(m, host, n, false, "icon_mlp_get_params");
}
int icon_mlp_get_grads(const icon_mlp_t* m, float* host, int64_t n) {
  return copy_out(m, host, n, true, "icon_mlp_get_grads");
}

int icon_mlp_forward(icon_mlp_t* m, const float* x, int32_t batch, float* y, void* stream) {
  if (!m || !x || !y) return fail_m(ICON_ERR_ARG, "icon_mlp_forward: NULL argument");
  int rc = check_batch(m, batch, "icon_mlp_forward");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = forward(m, x, batch, s);
  if (rc != ICON_OK) return rc;
  if (cudaMemcpy2DAsync(y, m->dims[3] * 4, m->y, m->lds[3] * 4, m->dims[3] * 4, batch, cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
    return fail_m(ICON_ERR_CUDA, "icon_mlp_forward: copy failed");
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_forward: ") + cudaGetErrorString(e));
  return tc_status("icon_mlp_forward");
}

int icon_mlp_backward(icon_mlp_t* m, const float* dy, int32_t batch, void* stream) {
  if (!m || !dy) return fail_m(ICON_ERR_ARG, "icon_mlp_backward: NULL argument");
  int rc = check_batch(m, batch, "icon_mlp_backward");
  if (rc) return rc;
  if (batch % 64) return fail_m(ICON_ERR_ARG, "icon_mlp_backward: batch must be a multiple of 64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpy2DAsync(m->dy, m->lds[3] * 4, dy, m->dims[3] * 4, m->dims[3] * 4, batch, cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
    return fail_m(ICON_ERR_CUDA, "icon_mlp_backward: copy failed");
  rc = backward(m, batch, s);
  if (rc != ICON_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_backward: ") + cudaGetErrorString(e));
  return tc_status("icon_mlp_backward");
}

int icon_mlp_adam(icon_mlp_t* m, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!m) return fail_m(ICON_ERR_ARG, "icon_mlp_adam: NULL argument");
  adam(m, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
  return ICON_OK;
}

int icon_mlp_train_step(icon_mlp_t* m, const float* x, const float* target, int32_t batch, float lr, double* loss,
                        void* stream) {
  if (!m || !x || !target) return fail_m(ICON_ERR_ARG, "icon_mlp_train_step: NULL argument");
  int rc = check_batch(m, batch, "icon_mlp_train_step");
  if (rc) return rc;
  if (batch % 64) return fail_m(ICON_ERR_ARG, "icon_mlp_train_step: batch must be a multiple of 64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = forward(m, x, batch, s);
  if (rc != ICON_OK) return rc;
  mlp_mse(batch, m->dims[3], m->y, m->lds[3], target, m->dims[3], m->dy, m->lds[3], m->rowloss, s);
  rc = backward(m, batch, s);
  if (rc != ICON_OK) return rc;
  adam(m, lr, 0.9f, 0.999f, 1e-8f, s);
  if (loss) {
    std::vector<double> rl(batch);
    if (cudaMemcpyAsync(rl.data(), m->rowloss, batch * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return fail_m(ICON_ERR_CUDA, "icon_mlp_train_step: copy failed");
    cudaStreamSynchronize(s);
    double t = 0.0;
    for (double v : rl) t += v;
    *loss = t / ((double)batch * m->dims[3]);
    rc = tc_status("icon_mlp_train_step");
    if (rc != ICON_OK) return rc;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_m(ICON_ERR_CUDA, std::string("icon_mlp_train_step: ") + cudaGetErrorString(e));
  return ICON_OK;
}

}  // extern "C"
