// Kernel launch interface of the dycore library (internal).
#pragma once
#include <cuda_bf16.h>
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

// Everything the stencil kernels of one precision mode need.
template <class T>
struct Ctx {
  GridT<T> g;
  VertT<T> v;
  ScalT<T> s;
  WorkT<T> w;
  TerrT<T> tr;   // terrain metrics (all null over flat ground)
  VaPatchT vp{};  // patches of the fused velocity advection (mixed precision, flat; n_patches 0: off)
};
// The fused velocity-advection kernel's shared-memory limit for these patches.
cudaError_t init_va_fused(const VaPatchT& pt);

// Device-side state of one dycore: FP64 factors and column-solve work, the
// FP32 mirrors (mixed mode) and the stencil context of the active mode.
// The mixed modes (FP32 stencils) differ only in the column solve's arithmetic.
inline bool is_mixed(int precision) { return precision != ICON_PREC_FP64; }

struct Engine {
  int precision = ICON_PREC_FP64;
  DevGrid g64{};
  DevVert v{};
  Scalars sc{};
  DevWork wk{};
  Mirrors m{};
  const double* rho_ref64 = nullptr;  // [nlev] rho offset of the mixed-mode perturbation
  Ctx<double> c64{};
  Ctx<float> c32{};
  // launch configuration picked by the autotuner: threads per CTA of each
  // stencil kernel (by kernel id) and the level-chunk depth of the column solve
  int threads[32] = {};
  // tile shape of the two-shape kernels (va_edge_pre, va_cell_w, sn_cell_div,
  // sn_edge_corr): 1 one warp per point (lanes over its levels), 0 one thread
  // per (point, level); -1 the compute type's default
  int shape[32] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                   -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
  int col_kc = 4;
  bool terrain = false;  // per-column heights: the terrain forms of the kernels
  // Host-array steps: when set, the first substep waits on this event right
  // after its predictor's velocity tendencies (which read only vn and w), so
  // that the copies of the other state fields overlap those kernels.
  cudaEvent_t io_wait = nullptr;
};

// Rows A1-A4 on (vn, w) in compute type T: writes ddt_vn [ne*nlev] and ddt_w
// [nc*(nlev+1)].  With divd2 != nullptr also the divergence-damping Laplacian
// of divd (A8).
// With terrain metrics in x.tr, the contravariant correction of vn goes to wcc
// (cells, half levels) and the advection uses w - wcc.
template <class T>
void launch_velocity_tendencies(const Ctx<T>& x, const T* vn, const T* w, T* ddt_vn, T* ddt_w, const T* divd,
                                T* divd2, cudaStream_t s, const int* threads = nullptr, T* wcc = nullptr,
                                const int* shapes = nullptr);
// Stencil kernel ids (index of Engine::threads) and their base names.
constexpr int kNumStencils = 16;
extern const char* const kStencilNames[kNumStencils];
// Fill n doubles with v (the autotuner's temporary state).
void launch_fill(double* p, size_t n, double v, cudaStream_t s);
// Event wait / record on s; inside a stream capture they become the graph's
// external event nodes.
void stream_wait_io(cudaStream_t s, cudaEvent_t e);
void stream_record_io(cudaStream_t s, cudaEvent_t e);
// Rows A5-A9: one predictor + corrector substep, state updated in place.
template <class T>
void launch_substep(const Engine& en, const Ctx<T>& x, const StateView& st, cudaStream_t s);
// Row A10: diffusion over dtime, state updated in place.
template <class T>
void launch_diffusion(const Engine& en, const Ctx<T>& x, const StateView& st, cudaStream_t s);
// Mixed mode: FP32 mirrors from the FP64 state.
void launch_refresh_mirrors(const Engine& en, const StateView& st, cudaStream_t s);
// Row A7: vertically implicit column solve (corrector = 0: the predicted state
// into en.wk.w_p/rho_p/theta_p; corrector = 1: the new state over st).
// Reads the flux divergences en.wk.div_m/div_t and ddt_w of type T.
template <class T>
void launch_column(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                   cudaStream_t s);
// The same over terrain: per-column metrics (en.v.colt) and the solve in
// w - wcc, wcc the contravariant correction (cells, half levels, type T).
template <class T>
void launch_column_terrain(const Engine& en, int corrector, const StateView& st, const T* ddt_w0, const T* ddt_w1,
                           const T* wcc, cudaStream_t s);
// Diagnostics: per-cell ps and T850 (either may be null), per-block partial
// column masses [diag_partials(nc)] and a non-finite flag (set to 1, never cleared).
int diag_partials(int nc);
void launch_diagnostics(const Engine& en, const double* area, const StateView& st, double* ps, double* t850,
                        double* partial, int* bad, cudaStream_t s);
// Learned corrector.  Column features (one thread per cell-level): raw FP32
// rows [nc][5 nlev] into raw (if given) and rows [nc][ldx] into x (normalised
// by mean/istd when given; the BF16 form always normalises: the network's
// input).  Edge features [ne][ldx] from the raw column features and vn.
// Increments of rows [row0, row0 + rows) applied to the state with per-block
// FP32 partial sums of the squared normalised outputs (apply_partials(n)
// blocks for n outputs); their two sums in FP64; training targets (plain -
// reduced).
void launch_col_features(const Engine& en, const StateView& st, float* raw, float* x, int ldx, const float* mean,
                         const float* istd, cudaStream_t s);
void launch_col_inputs(const Engine& en, const StateView& st, float* raw, __nv_bfloat16* x, int ldx,
                       const float* mean, const float* istd, cudaStream_t s);
void launch_edge_features(const Engine& en, const float* colx, const double* vn, float* x, int ldx,
                          const float* mean, const float* istd, cudaStream_t s);
void launch_edge_inputs(const Engine& en, const float* colx, const double* vn, __nv_bfloat16* x, int ldx,
                        const float* mean, const float* istd, cudaStream_t s);
int apply_partials(size_t n);
void launch_apply_col(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                      const float* stdv, const StateView& st, float* partial, cudaStream_t s);
void launch_apply_edge(const Engine& en, int row0, int rows, const float* y, int ldy, const float* mean,
                       const float* stdv, double* vn, float* partial, cudaStream_t s);
int reduce_stage_doubles();  // scratch doubles of launch_reduce_status
void launch_reduce_status(const float* partial, int n0, int n1, double* stage, double* out, cudaStream_t s);
void launch_targets(const Engine& en, const StateView& reduced, const StateView& plain, float* col_y, float* edge_y,
                    cudaStream_t s);
// nproma-blocked (ICON) <-> level-contiguous copy of one field of n points and
// nlev_x levels (to_blocked: library -> blocked).
void launch_blocked(bool to_blocked, int n, int nlev_x, int nproma, const double* src, double* dst, cudaStream_t s);
// One-time kernel attributes (dynamic shared memory above 48 KB).
cudaError_t init_column_kernels();
cudaError_t init_column_terrain_kernels();

}  // namespace icon
