// Row A7 over flat ground: launches of the column solve (kernel template in
// column_kernel.cuh) and the allocation-free entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>

#include "column_kernel.cuh"

namespace icon {

cudaError_t init_column_kernels() {
  cudaError_t e = init_col_forms<double, double, false>();
  if (e == cudaSuccess) e = init_col_forms<float, dws, false>();
  if (e == cudaSuccess) e = init_col_forms<float, double, false>();
  return e;
}

template <class T>
void launch_column(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                   cudaStream_t s) {
  const ColArgs<T> a = col_args<T>(en, corrector, st, ddt_w0, ddt_w1);
  constexpr bool mixed = std::is_same<T, float>::value;
  // the mixed step's solve: double-word FP32, or FP64 (ICON_PREC_MIXED_F64COL)
  const bool f64col = mixed && en.precision == ICON_PREC_MIXED_F64COL;
  const char* name = column_name(mixed, f64col, false, corrector);
  if (f64col)
    launch_col_form<T, double, false>(en, corrector, a, name, s);
  else
    launch_col_form<T, ColArith<T>, false>(en, corrector, a, name, s);
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
      cf[4] = q.dt_s * q.cpd * dref[k];
      cf[5] = q.dt_s * q.cpd * q.beta * inv_dzh[k];
      cf[6] = wgt[k];
      cf[7] = 1.0 - wgt[k];
      cf[3] = cf[6] * th_ref[k - 1] + cf[7] * th_ref[k];
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
  if (!(p->vwind_impl_wgt > 0.0 && p->vwind_impl_wgt <= 1.0))
    return report_error(ICON_ERR_ARG, std::string(fn) + "vwind_impl_wgt must be in (0, 1]");

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
  // the levels noalloc_metrics may damp (an upper bound: ray_fac is 1 below)
  v.n_ray = 0;
  if (p->rayleigh_coeff > 0.0)
    for (int k = 0; k <= nlev; ++k)
      if (z_ifc[k] > p->damp_height) v.n_ray = k + 1;
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
