// Kernel launch interface of the dycore library (internal).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace icon {

// Optional per-launch timing: when `g_prof` is set on the launching thread,
// every kernel launch is bracketed by a CUDA event pair on its stream.
struct Prof {
  struct Rec {
    const char* name;
    cudaEvent_t e0, e1;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  ~Prof() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};
extern thread_local Prof* g_prof;

#define ICON_LAUNCH_SMEM(name, grid, block, smem, stream, kernel, ...) \
  do {                                                                  \
    cudaEvent_t e0_ = nullptr;                                          \
    if (g_prof) {                                                       \
      e0_ = g_prof->get();                                              \
      cudaEventRecord(e0_, stream);                                     \
    }                                                                   \
    kernel<<<grid, block, smem, stream>>>(__VA_ARGS__);                 \
    if (g_prof) {                                                       \
      cudaEvent_t e1_ = g_prof->get();                                  \
      cudaEventRecord(e1_, stream);                                     \
      g_prof->recs.push_back({name, e0_, e1_});                         \
    }                                                                   \
  } while (0)
#define ICON_LAUNCH(name, grid, block, stream, kernel, ...) \
  ICON_LAUNCH_SMEM(name, grid, block, 0, stream, kernel, __VA_ARGS__)

// Device pointers of one prognostic state (level-contiguous, FP64).
struct StateView {
  double *vn, *w, *rho, *exner, *theta_v, *exner_pr;
};

// Rows A1-A4 on (vn, w): writes ddt_vn [ne*nlev] and ddt_w [nc*(nlev+1)].
// With divd2 != nullptr also the divergence-damping Laplacian of divd (A8).
void launch_velocity_tendencies(const DevGrid& g, const DevVert& v, const double* vn, const double* w,
                                DevWork& wk, double* ddt_vn, double* ddt_w, const double* divd,
                                double* divd2, cudaStream_t s);
// Rows A5-A9: one predictor + corrector substep, state updated in place.
void launch_substep(const DevGrid& g, const DevVert& v, const Scalars& sc, const StateView& st, DevWork& wk,
                    cudaStream_t s);
// Row A7: vertically implicit column solve (predictor: corrector = 0 writes the
// predicted state to wk.w_p/rho_p/exner_p/theta_p; corrector = 1 writes the new
// state over st).  Needs wk.div_m/div_t (flux divergences) of the pass.
void launch_column(const DevGrid& g, const DevVert& v, const Scalars& sc, int corrector, const StateView& st,
                   DevWork& wk, cudaStream_t s);
// One-time kernel attributes (dynamic shared memory above 48 KB).
cudaError_t init_column_kernels();

// Row A10: diffusion over dtime, state updated in place.
void launch_diffusion(const DevGrid& g, const DevVert& v, const Scalars& sc, const StateView& st, DevWork& wk,
                      cudaStream_t s);

}  // namespace icon
