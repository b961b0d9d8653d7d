// Diagnostics of a state (outside the timed step): surface pressure, 850 hPa
// temperature, total mass, and a check for non-finite values.
//   ps: exner at the ground extrapolated hydrostatically from the lowest full
//       level with its theta_v, ps = p00 exner_sfc^(cpd/rd);
//   T850: linear interpolation of T = theta_v exner in ln p between the two
//       levels around 850 hPa (the lowest level's T if the column is above);
//   mass: sum_c A_c sum_k rho dz_k, reduced in a fixed order (no atomics).
#include <cuda_runtime.h>

#include "kernels.h"

namespace icon {
namespace {

constexpr int kDiagThreads = 256;

// dz_c: per-column layer thicknesses over terrain (NULL: the per-level dz)
__global__ void diag_columns(int nc, int nlev, const double* __restrict__ dz, const double* __restrict__ dz_c,
                             const double* __restrict__ area,
                             double grav, double cpd, double rd, double p00, const double* __restrict__ w,
                             const double* __restrict__ rho, const double* __restrict__ exner,
                             const double* __restrict__ theta, double* __restrict__ ps, double* __restrict__ t850,
                             double* __restrict__ partial, int* __restrict__ bad) {
  __shared__ double red[kDiagThreads];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (c < nc) {
    const double* ex = exner + (size_t)c * nlev;
    const double* th = theta + (size_t)c * nlev;
    const double* r = rho + (size_t)c * nlev;
    const double* wc = w + (size_t)c * (nlev + 1);
    const double* dzk = dz_c ? dz_c + (size_t)c * nlev : dz;
    bool finite = true;
    for (int k = 0; k < nlev; ++k) {
      finite = finite && isfinite(ex[k]) && isfinite(th[k]) && isfinite(r[k]) && isfinite(wc[k]);
      m += r[k] * dzk[k];
    }
    finite = finite && isfinite(wc[nlev]);
    if (!finite) atomicOr(bad, 1);
    m *= area[c];
    const double kappa_inv = cpd / rd;
    const double z_low = 0.5 * dzk[nlev - 1];  // the lowest full level, dz/2 above the ground
    const double ex_sfc = ex[nlev - 1] + grav * z_low / (cpd * th[nlev - 1]);
    if (ps) ps[c] = p00 * pow(ex_sfc, kappa_inv);
    if (t850) {
      const double target = 85000.0;
      double t = th[nlev - 1] * ex[nlev - 1];
      double p_lo = p00 * pow(ex[nlev - 1], kappa_inv);
      for (int k = nlev - 1; k > 0; --k) {
        const double p_up = p00 * pow(ex[k - 1], kappa_inv);
        if (p_lo >= target && target > p_up) {
          const double x = (log(target) - log(p_lo)) / (log(p_up) - log(p_lo));
          const double t_lo = th[k] * ex[k], t_up = th[k - 1] * ex[k - 1];
          t = t_lo + x * (t_up - t_lo);
          break;
        }
        p_lo = p_up;
      }
      t850[c] = t;
    }
  }
  // fixed-order tree reduction of the column masses within the block
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void diag_finite(size_t n, const double* __restrict__ x, int* __restrict__ bad) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicOr(bad, 1);
}

}  // namespace

int diag_partials(int nc) { return (nc + kDiagThreads - 1) / kDiagThreads; }

void launch_diagnostics(const Engine& en, const double* area, const StateView& st, double* ps, double* t850,
                        double* partial, int* bad, cudaStream_t s) {
  const int nc = en.g64.nc, nlev = en.v.nlev;
  ICON_LAUNCH("diag_columns", (unsigned)diag_partials(nc), kDiagThreads, s, diag_columns, nc, nlev, en.v.dz, en.v.dz_c, area,
              en.sc.grav, en.sc.cpd, en.sc.rd, en.sc.p00, st.w, st.rho, st.exner, st.theta_v, ps, t850, partial,
              bad);
  const size_t nvn = (size_t)en.g64.ne * nlev;
  ICON_LAUNCH("diag_finite", (unsigned)((nvn + 255) / 256), 256, s, diag_finite, nvn, st.vn, bad);
}

}  // namespace icon
