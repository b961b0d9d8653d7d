// C-ABI entry points of the dycore library (paper Sec. 4.3: the host model
// gathers field pointers and calls a C function; scalars by value, arrays by
// reference without copies, device arrays accepted directly).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "mlp.h"

using namespace icon;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

namespace icon {
int report_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace icon

namespace {

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t err_ = (expr);                                                              \
    if (err_ != cudaSuccess)                                                                \
      return fail(ICON_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(err_));     \
  } while (0)

// Owner of a set of device allocations.
struct DevArena {
  std::vector<void*> ptrs;
  cudaError_t status = cudaSuccess;
  template <typename T>
  T* upload(const std::vector<T>& h) {
    T* d = alloc<T>(h.size());
    if (d && !h.empty()) {
      cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) status = e;
    }
    return d;
  }
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (status != cudaSuccess) return nullptr;
    cudaError_t e = cudaMalloc(&p, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
      status = e;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

}  // namespace

struct icon_grid {
  HostGrid host;
  DevGrid dev{};
  DevArena arena;
};

struct GraphEntry {
  StateView key{};
  bool io = false;  // captured with the host-copy events (staging state of a host-array step)
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
};

struct icon_dycore {
  const icon_grid* grid = nullptr;
  icon_dycore_params_t params{};
  Scalars sc{};
  int nlev = 0;
  std::vector<double> z_ifc, theta_ref, exner_ref;
  Engine en;
  DevArena arena;
  cudaStream_t stream = nullptr;       // caller's stream (may be the default stream)
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  GraphEntry graphs[2];
  unsigned long long use_counter = 0;
  StateView staging{};                 // device copy used when the caller passes host arrays
  bool have_staging = false;
  // host-array steps: a private stream for the copies of the fields the step
  // reads late or finishes early, and the events that order them with the step
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_start = nullptr, io_in = nullptr, io_out = nullptr;
  // learned corrector (allocated on first use): saved input state, features, norm partials
  StateView saved{};
  float* colx = nullptr;                                  // raw column features [nc][5 nlev]
  __nv_bfloat16 *col16 = nullptr, *edge16 = nullptr;     // network inputs [nc][ld_col16], [ne][ld_edge16]
  int ld_col16 = 0, ld_edge16 = 0;
  float* partial = nullptr;
  double* status = nullptr;
  int partial_cap = 0;
};

extern "C" {

const char* icon_last_error(void) { return g_last_error.c_str(); }

void icon_dycore_params_default(icon_dycore_params_t* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->dtime = 1800.0;
  p->ndyn_substeps = 5;
  p->grav = 9.80665;
  p->rd = 287.04;
  p->cpd = 1004.64;
  p->p00 = 1.0e5;
  p->omega = 7.29212e-5;
  p->vwind_impl_wgt = 0.65;
  p->wgt_nnow_vel = 0.25;
  p->wgt_nnew_vel = 0.75;
  p->wgt_nnow_rth = 0.6;
  p->wgt_nnew_rth = 0.4;
  p->exner_exfac = 1.0 / 3.0;
  p->divdamp_fac = 0.0025;
  p->divflux_fac = 0.07;
  p->rayleigh_coeff = 0.0;
  p->damp_height = 20000.0;
  p->hdiff_smag_fac = 0.015;
  p->hdiff_k4 = 1.0 / 288.0;
  p->hdiff_w_k4 = 1.0 / 288.0;
  p->hdiff_temp = 1;
  p->ref_T0 = 250.0;
  p->precision = ICON_PREC_FP64;
  p->use_graph = 1;
  p->autotune = 1;
  p->synchronous = 1;
  p->stream = nullptr;
  p->column_chunk = 0;
  p->steep_hpg = 0;
  p->hdiff_tenh_fac = 0.0;
  p->hdiff_tenh_thresh = 5.0;
  p->hdiff_tenh_levels = 5;
  p->fused_advection = 0;
}

int icon_grid_create(const icon_grid_desc_t* d, icon_grid_t** out) {
  if (!d || !out) return fail(ICON_ERR_ARG, "icon_grid_create: NULL argument");
  *out = nullptr;
  if (d->n_cells <= 0 || d->n_edges <= 0 || d->n_verts <= 0)
    return fail(ICON_ERR_ARG, "icon_grid_create: counts must be positive");
  if (d->index_base != 0 && d->index_base != 1)
    return fail(ICON_ERR_ARG, "icon_grid_create: index_base must be 0 or 1");
  if (!d->c2v || !d->c2e || !d->e2c || !d->e2v || !d->v2e || !d->v2c || !d->cell_xyz || !d->vert_xyz ||
      !d->edge_xyz)
    return fail(ICON_ERR_ARG, "icon_grid_create: NULL table or coordinate pointer");
  icon_grid* g = new (std::nothrow) icon_grid();
  if (!g) return fail(ICON_ERR_ARG, "icon_grid_create: out of host memory");
  std::string err = build_host_grid(d, &g->host);
  if (!err.empty()) {
    delete g;
    return fail(ICON_ERR_GRID, "icon_grid_create: " + err);
  }
  const HostGrid& h = g->host;
  DevGrid& v = g->dev;
  DevArena& A = g->arena;
  v.nc = h.nc;
  v.ne = h.ne;
  v.nv = h.nv;
  v.c2e = A.upload(h.c2e);
  v.c2e2c = A.upload(h.c2e2c);
  v.e2c = A.upload(h.e2c);
  v.e2v = A.upload(h.e2v_t);
  v.e2c2v = A.upload(h.e2c2v);
  v.e2c2e = A.upload(h.e2c2e);
  v.v2e = A.upload(h.v2e);
  v.v2c = A.upload(h.v2c);
  v.div_c = A.upload(h.div_c);
  {
    std::vector<float> hl(2 * h.div_c.size());
    for (size_t i = 0; i < h.div_c.size(); ++i) split_hl(h.div_c[i], &hl[2 * i]);
    v.div_c_hl = A.upload(hl);
  }
  v.lap_c = A.upload(h.lap_c);
  v.e2c_w = A.upload(h.e2c_w);
  v.grad_c = A.upload(h.grad_c);
  v.inv_d = A.upload(h.inv_d);
  v.inv_l = A.upload(h.inv_l);
  v.vt_w = A.upload(h.vt_w);
  v.upw = A.upload(h.upw);
  v.nt = A.upload(h.nt);
  v.inv_dn = A.upload(h.inv_dn);
  v.curl_v = A.upload(h.curl_v);
  v.c2v_w = A.upload(h.c2v_w);
  v.uv_w = A.upload(h.uv_w);
  v.mean_area = h.mean_area;
  v.cell_area = A.upload(h.cell_area);
  v.uv_c = A.upload(std::vector<float>(h.uv_c.begin(), h.uv_c.end()));
  if (A.status != cudaSuccess) {
    std::string m = std::string("icon_grid_create: ") + cudaGetErrorString(A.status);
    A.release();
    delete g;
    return fail(ICON_ERR_CUDA, m);
  }
  *out = g;
  return ICON_OK;
}

int icon_grid_destroy(icon_grid_t* g) {
  if (!g) return ICON_OK;
  g->arena.release();
  delete g;
  return ICON_OK;
}

static void free_graphs(icon_dycore* d) {
  for (auto& e : d->graphs) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    e = GraphEntry{};
  }
}

}  // extern "C"

namespace {

void enqueue_op(icon_dycore* d, int op, const StateView& st, cudaStream_t s);

// The dycore's own stream for graph capture.
void release_streams(icon_dycore* d) {
  if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
  d->cap_stream = nullptr;
}

// The common part of icon_dycore_create and icon_dycore_create_terrain:
// z_ifc [nlev+1] the heights the per-level tables use (column 0's over
// terrain), z_cols [nc*(nlev+1)] the per-column heights (NULL: flat ground).
int create_dycore(const icon_grid_t* grid, int nlev, const double* z_ifc, const double* z_cols,
                  const icon_dycore_params_t* p, icon_dycore_t** out, const char* fn);

// Autotuner: time every kernel of one step on a temporary uniform state with
// each candidate launch shape (CUDA events around every launch) and keep the
// fastest shape per kernel.
// Every coefficient and work pointer the kernels of the active precision
// dereference must be set: a missing one is an internal error reported at
// create, never a device fault.
template <class T>
bool grid_complete(const GridT<T>& g) {
  const void* p[] = {g.c2e, g.c2e2c, g.e2c, g.e2v, g.e2c2v, g.e2c2e, g.v2e, g.v2c, g.div_c, g.lap_c, g.e2c_w,
                     g.grad_c, g.k4w_c, g.inv_d, g.inv_l, g.f_e, g.vt_w, g.upw, g.nt, g.inv_dn, g.smag_a, g.k4_a,
                     g.fdiv_e, g.ddamp_e, g.curl_v, g.c2v_w, g.uv_w, g.cell_area, g.uv_c, g.div_c_hl,
                     g.upw_s, g.cpd_inv_d, g.hinv_d, g.d_o_l, g.grad_s, g.lap_s, g.e2c_wd};
  for (const void* q : p)
    if (!q) return false;
  return true;
}

template <class T>
bool terrain_complete(const TerrT<T>& t) {
  const void* p[] = {t.wgt_e, t.qdz_e, t.ddxn_ifc, t.ddxt_ifc, t.ddxn_mc, t.qdzh_c, t.inv_dzm_c, t.fx_ratio,
                     t.wcc0, t.wcc1};
  for (const void* q : p)
    if (!q) return false;
  return true;
}

bool work_complete(const DevWork& w) {
  const void* p[] = {w.div_m, w.div_t, w.rho_p, w.theta_p, w.w_p, w.pex, w.col, w.zbl, w.diag, w.flag};
  for (const void* q : p)
    if (!q) return false;
  return true;
}

int autotune(icon_dycore* d) {
  const HostGrid& h = d->grid->host;
  const size_t nlev = d->nlev, ef = h.ne * nlev, cf = h.nc * nlev, ch = h.nc * (nlev + 1);
  StateView st{};
  double** fields[6] = {&st.vn, &st.w, &st.rho, &st.exner, &st.theta_v, &st.exner_pr};
  const size_t sizes[6] = {ef, ch, cf, cf, cf, cf};
  const double values[6] = {10.0, 0.0, 1.0, 0.9, 300.0, 0.0};
  int rc = ICON_OK;
  for (int i = 0; i < 6 && rc == ICON_OK; ++i) {
    cudaError_t e = cudaMalloc(fields[i], sizes[i] * sizeof(double));
    if (e != cudaSuccess) {
      *fields[i] = nullptr;
      rc = fail(ICON_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    } else {
      launch_fill(*fields[i], sizes[i], values[i], d->stream);
    }
  }
  // Candidates: threads per CTA (128, 256, 512) x tile shape (one thread per
  // (point, level), or one warp per point with its lanes over the levels) for
  // the stencil kernels; levels per shared-memory chunk (8, 6, 4) for the
  // column solve.  Each candidate runs kReps steps; a kernel's time is the
  // smallest of its per-step sums, so a single noisy sample cannot decide.
  constexpr int kReps = 3;
  const int cand[3] = {128, 256, 512};
  constexpr double kInf = 1e300;
  // t[k][shape][ci]: best per-step time of stencil kernel k
  std::vector<double> t(kNumStencils * 2 * 3, kInf);
  auto tk = [&](int k, int sh, int ci) -> double& { return t[((size_t)k * 2 + sh) * 3 + ci]; };
  const int col_cand[3] = {8, 6, 4};
  double col_t[3] = {kInf, kInf, kInf};
  auto run = [&](int ci, int shape, int kc, bool stencils) -> int {
    for (int k = 0; k < kNumStencils; ++k) {
      d->en.threads[k] = cand[ci];
      d->en.shape[k] = shape;
    }
    d->en.col_kc = kc;
    Prof prof;
    g_prof = &prof;
    enqueue_op(d, 0, st, d->stream);
    g_prof = nullptr;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    std::vector<double> sum(kNumStencils, 0.0);
    double col = 0.0;
    for (const auto& r : prof.recs) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, r.e0, r.e1));
      std::string nm = r.name;
      if (nm.compare(0, 9, "sn_column") == 0) {
        col += ms;
        continue;
      }
      if (nm.compare(0, 15, "sn_cell_fluxsum") == 0) nm = "sn_cell_fluxdiv" + nm.substr(15);  // same id
      for (int k = 0; k < kNumStencils; ++k) {
        const std::string base = kStencilNames[k];
        if (nm == base || nm == base + "_f32" || nm == base + "_terrain" || nm == base + "_terrain_f32")
          sum[k] += ms;
      }
    }
    if (stencils)
      for (int k = 0; k < kNumStencils; ++k)
        if (sum[k] > 0.0) tk(k, shape, ci) = std::min(tk(k, shape, ci), sum[k]);
    for (int j = 0; j < 3; ++j)
      if (col_cand[j] == kc) col_t[j] = std::min(col_t[j], col);
    return ICON_OK;
  };
  if (rc == ICON_OK) rc = run(1, 0, 8, false);  // warm-up (module load, first-touch)
  if (rc == ICON_OK) col_t[0] = kInf;
  for (int shape = 0; shape < 2; ++shape)
    for (int ci = 0; ci < 3; ++ci)
      for (int r = 0; r < kReps && rc == ICON_OK; ++r) rc = run(ci, shape, 8, true);
  for (int j = 1; j < 3; ++j)
    for (int r = 0; r < kReps && rc == ICON_OK; ++r) rc = run(1, 0, col_cand[j], false);
  for (double* p : {st.vn, st.w, st.rho, st.exner, st.theta_v, st.exner_pr})
    if (p) cudaFree(p);
  if (rc != ICON_OK) return rc;
  for (int k = 0; k < kNumStencils; ++k) {
    int best_sh = 0, best_ci = 1;
    for (int sh = 0; sh < 2; ++sh)
      for (int ci = 0; ci < 3; ++ci)
        if (tk(k, sh, ci) < tk(k, best_sh, best_ci)) {
          best_sh = sh;
          best_ci = ci;
        }
    d->en.threads[k] = cand[best_ci];
    // only va_edge_pre, va_cell_w, sn_cell_div and sn_edge_corr have both shapes
    d->en.shape[k] = (k == 0 || k == 3 || k == 6 || k == 8) ? best_sh : -1;
  }
  int best_kc = 0;
  for (int j = 1; j < 3; ++j)
    if (col_t[j] < col_t[best_kc]) best_kc = j;
  d->en.col_kc = col_cand[best_kc];
  return ICON_OK;
}

}  // namespace

extern "C" {

int icon_dycore_create(const icon_grid_t* grid, int32_t nlev, const double* z_ifc,
                       const icon_dycore_params_t* p, icon_dycore_t** out) {
  if (!grid || !z_ifc || !p || !out) return fail(ICON_ERR_ARG, "icon_dycore_create: NULL argument");
  *out = nullptr;
  if (nlev < 2) return fail(ICON_ERR_ARG, "icon_dycore_create: nlev must be >= 2");
  for (int k = 0; k <= nlev; ++k)
    if (!std::isfinite(z_ifc[k])) return fail(ICON_ERR_ARG, "icon_dycore_create: z_ifc not finite");
  for (int k = 0; k < nlev; ++k)
    if (!(z_ifc[k] > z_ifc[k + 1])) return fail(ICON_ERR_ARG, "icon_dycore_create: z_ifc must decrease");
  if (z_ifc[nlev] != 0.0) return fail(ICON_ERR_ARG, "icon_dycore_create: z_ifc[nlev] must be 0 (flat ground)");
  return create_dycore(grid, nlev, z_ifc, nullptr, p, out, "icon_dycore_create");
}

int icon_dycore_create_terrain(const icon_grid_t* grid, int32_t nlev, const double* z_ifc,
                               const icon_dycore_params_t* p, icon_dycore_t** out) {
  if (!grid || !z_ifc || !p || !out) return fail(ICON_ERR_ARG, "icon_dycore_create_terrain: NULL argument");
  *out = nullptr;
  if (nlev < 2) return fail(ICON_ERR_ARG, "icon_dycore_create_terrain: nlev must be >= 2");
  return create_dycore(grid, nlev, z_ifc, z_ifc, p, out, "icon_dycore_create_terrain");
}

}  // extern "C"

namespace {

int create_dycore(const icon_grid_t* grid, int nlev, const double* z_ifc, const double* z_cols,
                  const icon_dycore_params_t* p, icon_dycore_t** out, const char* fn) {
  const std::string fname = fn;
  if (!(p->dtime > 0.0) || p->ndyn_substeps < 1)
    return fail(ICON_ERR_ARG, fname + ": dtime must be > 0 and ndyn_substeps >= 1");
  if (p->precision != ICON_PREC_FP64 && p->precision != ICON_PREC_MIXED && p->precision != ICON_PREC_MIXED_F64COL)
    return fail(ICON_ERR_ARG, fname + ": precision must be ICON_PREC_FP64, ICON_PREC_MIXED or ICON_PREC_MIXED_F64COL");
  if (!(p->vwind_impl_wgt > 0.0 && p->vwind_impl_wgt <= 1.0))
    return fail(ICON_ERR_ARG, fname + ": vwind_impl_wgt must be in (0, 1]");
  if (p->column_chunk != 0 && p->column_chunk != 4 && p->column_chunk != 6 && p->column_chunk != 8)
    return fail(ICON_ERR_ARG, fname + ": column_chunk must be 0, 4, 6 or 8");
  if (!(p->hdiff_tenh_fac >= 0.0) || (p->hdiff_tenh_fac > 0.0 && !(p->hdiff_tenh_thresh > 0.0)) ||
      p->hdiff_tenh_levels < 0)
    return fail(ICON_ERR_ARG, fname + ": enhanced temperature diffusion needs fac >= 0, thresh > 0, levels >= 0");
  if (p->steep_hpg && nlev < 3) return fail(ICON_ERR_ARG, fname + ": steep_hpg needs nlev >= 3");
  // terrain: every column validated and its metrics derived before any allocation
  HostTerrain ht;
  if (z_cols) {
    Scalars s0{};
    s0.dt_s = p->dtime / p->ndyn_substeps;
    s0.beta = p->vwind_impl_wgt;
    s0.rd_o_cvd = p->rd / (p->cpd - p->rd);
    std::string err = build_terrain(grid->host, nlev, z_cols, *p, s0, &ht);
    if (!err.empty()) return fail(ICON_ERR_ARG, fname + ": " + err);
  }

  icon_dycore* d = new (std::nothrow) icon_dycore();
  if (!d) return fail(ICON_ERR_ARG, fname + ": out of host memory");
  d->grid = grid;
  d->params = *p;
  d->nlev = nlev;
  d->stream = static_cast<cudaStream_t>(p->stream);
  const HostGrid& h = grid->host;
  const int nc = h.nc, ne = h.ne, nv = h.nv;

  // scalars
  Scalars& s = d->sc;
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
  s.divflux = p->divflux_fac * h.mean_area;
  s.rd_o_cvd = p->rd / s.cvd;
  s.cvd_o_rd = s.cvd / p->rd;
  s.hdiff_temp = p->hdiff_temp ? 1 : 0;

  // vertical metrics and reference state (row A0); over terrain those of
  // column 0, which serve as the mixed mode's FP32 perturbation offsets
  d->z_ifc.assign(z_ifc, z_ifc + nlev + 1);
  ColumnMetrics cm0;
  column_metrics(z_ifc, nlev, *p, s, &cm0);
  std::vector<double>& dz = cm0.dz;
  std::vector<double>& inv_dz = cm0.inv_dz;
  std::vector<double>& inv_dzh = cm0.inv_dzh;
  std::vector<double>& wgt = cm0.wgt;
  std::vector<double>& dref = cm0.dref;
  std::vector<double>& ray = cm0.ray;
  std::vector<double>& colc = cm0.colc;
  d->theta_ref = cm0.theta_ref;
  d->exner_ref = cm0.exner_ref;
  // reference density: the offset of the FP32 rho perturbation (mixed mode)
  std::vector<double> rho_ref(nlev);
  for (int k = 0; k < nlev; ++k)
    rho_ref[k] = p->p00 * std::pow(d->exner_ref[k], s.cvd / p->rd) / (p->rd * d->theta_ref[k]);

  DevArena& A = d->arena;
  Engine& en = d->en;
  en.precision = p->precision;
  DevVert& v = en.v;
  v.nlev = nlev;
  v.dz = A.upload(dz);
  v.inv_dz = A.upload(inv_dz);
  v.inv_dzh = A.upload(inv_dzh);
  v.wgt = A.upload(wgt);
  v.theta_ref = A.upload(d->theta_ref);
  v.exner_ref = A.upload(d->exner_ref);
  v.dexner_ref_ic = A.upload(dref);
  v.ray_fac = A.upload(ray);
  v.n_ray = 0;
  for (int k = 0; k <= nlev; ++k)
    if (ray[k] != 1.0) v.n_ray = k + 1;
  v.colc = A.upload(colc);
  v.lev_hl = A.upload(level_pairs(nlev, colc.data(), d->exner_ref.data(), d->theta_ref.data(), dz.data(), ray.data(),
                                  rho_ref.data()));
  v.lev64 = A.upload(level_table64(nlev, colc.data(), d->exner_ref.data(), d->theta_ref.data(), dz.data(), ray.data(),
                                   rho_ref.data()));
  en.rho_ref64 = A.upload(rho_ref);
  en.sc = s;

  // parameter-dependent grid factors
  std::vector<double> fe(ne), smag(ne), k4(ne), k4w(nc), fdiv(ne), ddamp(ne);
  for (int e = 0; e < ne; ++e) {
    fe[e] = 2.0 * p->omega * h.coriolis_z[e];
    smag[e] = p->hdiff_smag_fac * h.edge_area[e];
    k4[e] = p->hdiff_k4 * h.edge_area[e] * h.edge_area[e];
    fdiv[e] = s.divflux * h.inv_d[e];
    ddamp[e] = s.divdamp * h.mean_area * h.mean_area * h.inv_d[e];
  }
  for (int c = 0; c < nc; ++c) k4w[c] = p->hdiff_w_k4 * h.cell_area[c] * h.cell_area[c];
  // dycore-level factors of the predictor's edge kernel: upwind offsets with
  // the half-substep scaling folded in, and cpd / d_e
  std::vector<double> upw_s(h.upw), cid(ne), tenh(ne);
  for (int e = 0; e < ne; ++e) tenh[e] = p->hdiff_tenh_fac * h.edge_area[e] / p->dtime;
  const bool tenh_on = p->hdiff_temp && p->hdiff_tenh_fac > 0.0 && p->hdiff_tenh_levels > 0;
  for (int e = 0; e < ne; ++e) {
    for (int side = 0; side < 2; ++side)
      for (int j = 2; j < 6; ++j) upw_s[12 * (size_t)e + 6 * side + j] *= 0.5 * s.dt_s;
    cid[e] = p->cpd * h.inv_d[e];
  }
  // factors that fold constants of the stencils into stored products (fewer
  // FP64 operations per point-level)
  std::vector<double> hinv_d(ne), d_o_l(ne), grad_s(2 * (size_t)nc, 0.0), lap_s(nc, 0.0), e2c_wd(3 * (size_t)nc);
  for (int e = 0; e < ne; ++e) {
    hinv_d[e] = 0.5 * h.inv_d[e];
    d_o_l[e] = h.inv_l[e] / h.inv_d[e];
  }
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < 3; ++j) {
      const size_t cj = 3 * (size_t)c + j;
      grad_s[2 * (size_t)c] += h.grad_c[2 * cj];
      grad_s[2 * (size_t)c + 1] += h.grad_c[2 * cj + 1];
      lap_s[c] += h.lap_c[cj];
      e2c_wd[cj] = h.e2c_w[cj] * h.inv_d[h.c2e[cj]];
    }
  en.g64 = grid->dev;
  en.g64.hinv_d = A.upload(hinv_d);
  en.g64.d_o_l = A.upload(d_o_l);
  en.g64.grad_s = A.upload(grad_s);
  en.g64.lap_s = A.upload(lap_s);
  en.g64.e2c_wd = A.upload(e2c_wd);
  en.g64.upw_s = A.upload(upw_s);
  en.g64.cpd_inv_d = A.upload(cid);
  en.g64.tenh_a = tenh_on ? A.upload(tenh) : nullptr;
  en.g64.f_e = A.upload(fe);
  en.g64.smag_a = A.upload(smag);
  en.g64.k4_a = A.upload(k4);
  en.g64.k4w_c = A.upload(k4w);
  en.g64.fdiv_e = A.upload(fdiv);
  en.g64.ddamp_e = A.upload(ddamp);

  const size_t ef = (size_t)ne * nlev, eh = (size_t)ne * (nlev + 1);
  const size_t cf = (size_t)nc * nlev, ch = (size_t)nc * (nlev + 1);
  const size_t vf = (size_t)nv * nlev, vh = (size_t)nv * (nlev + 1);
  auto build_ctx = [&](auto& x, auto tag) {
    using T = decltype(tag);
    auto up = [&](const std::vector<double>& src) { return A.upload(std::vector<T>(src.begin(), src.end())); };
    GridT<T>& g = x.g;
    const DevGrid& g0 = grid->dev;
    g.nc = nc;
    g.ne = ne;
    g.nv = nv;
    g.c2e = g0.c2e;
    g.c2e2c = g0.c2e2c;
    g.e2c = g0.e2c;
    g.e2v = g0.e2v;
    g.e2c2v = g0.e2c2v;
    g.e2c2e = g0.e2c2e;
    g.v2e = g0.v2e;
    g.v2c = g0.v2c;
    g.div_c = up(h.div_c);
    g.lap_c = up(h.lap_c);
    g.e2c_w = up(h.e2c_w);
    g.grad_c = up(h.grad_c);
    g.k4w_c = up(k4w);
    g.inv_d = up(h.inv_d);
    g.inv_l = up(h.inv_l);
    g.hinv_d = up(hinv_d);
    g.d_o_l = up(d_o_l);
    g.grad_s = up(grad_s);
    g.lap_s = up(lap_s);
    g.e2c_wd = up(e2c_wd);
    g.f_e = up(fe);
    g.vt_w = up(h.vt_w);
    g.upw = up(h.upw);
    g.upw_s = up(upw_s);
    g.cpd_inv_d = up(cid);
    g.tenh_a = tenh_on ? up(tenh) : nullptr;
    g.nt = up(h.nt);
    g.inv_dn = up(h.inv_dn);
    g.smag_a = up(smag);
    g.k4_a = up(k4);
    g.fdiv_e = up(fdiv);
    g.ddamp_e = up(ddamp);
    g.curl_v = up(h.curl_v);
    g.c2v_w = up(h.c2v_w);
    g.uv_w = up(h.uv_w);
    g.div_c_hl = g0.div_c_hl;
    g.cell_area = g0.cell_area;
    g.uv_c = g0.uv_c;
    g.mean_area = (T)h.mean_area;
    VertT<T>& vt = x.v;
    vt.nlev = nlev;
    vt.inv_dz = up(inv_dz);
    vt.inv_dzh = up(inv_dzh);
    {
      std::vector<double> q(inv_dz), qh(inv_dzh);
      for (double& x : q) x *= 0.25;
      for (double& x : qh) x *= 0.5;
      vt.qdz = up(q);
      vt.qdzh = up(qh);
    }
    vt.wgt = up(wgt);
    vt.theta_ref = up(d->theta_ref);
    vt.rho_ref = up(rho_ref);
    vt.exner_ref = v.exner_ref;
    ScalT<T>& st = x.s;
    st.dt_s = (T)s.dt_s;
    st.dtime = (T)s.dtime;
    st.cpd = (T)s.cpd;
    st.exfac = (T)s.exfac;
    st.divdamp = (T)s.divdamp;
    st.divflux = (T)s.divflux;
    st.wnow_vel = (T)s.wnow_vel;
    st.wnew_vel = (T)s.wnew_vel;
    st.hdiff_temp = s.hdiff_temp;
    st.tenh_levels = tenh_on ? std::min(p->hdiff_tenh_levels, nlev) : 0;  // more levels than the column: all
    st.tenh_thresh = (T)p->hdiff_tenh_thresh;
    WorkT<T>& w = x.w;
    w.vt = A.template alloc<T>(ef);
    w.ekin_e = A.template alloc<T>(ef);
    w.ddt_vn0 = A.template alloc<T>(ef);
    w.ddt_vn1 = A.template alloc<T>(ef);
    w.rho_e = A.template alloc<T>(ef);
    w.theta_e = A.template alloc<T>(ef);
    w.hpg = A.template alloc<T>(ef);
    w.vn_p = A.template alloc<T>(ef);
    w.lap_vn = A.template alloc<T>(ef);
    w.nu = A.template alloc<T>(ef);
    w.gw_e = A.template alloc<T>(eh);
    w.vn_ie = A.template alloc<T>(eh);
    if constexpr (std::is_same<T, double>::value) {
      w.flx_m = A.template alloc<T>(ef);
      w.flx_t = A.template alloc<T>(ef);
    }
    w.ekin_c = A.template alloc<T>(cf);
    w.grad4 = A.template alloc<T>(4 * cf);
    w.divd = A.template alloc<T>(cf);
    w.divd2 = A.template alloc<T>(cf);
    w.dtheta = A.template alloc<T>(cf);
    w.div_l = A.template alloc<T>(cf);
    w.div_vn = A.template alloc<T>(cf);
    w.wq = A.template alloc<T>(cf);
    w.tenh_ex = tenh_on ? A.template alloc<T>(cf) : nullptr;
    w.ddt_w0 = A.template alloc<T>(ch);
    w.ddt_w1 = A.template alloc<T>(ch);
    w.lap_w = A.template alloc<T>(ch);
    w.zeta = A.template alloc<T>(vf);
    w.uv3 = A.template alloc<T>(3 * vf);
    w.curl_l = A.template alloc<T>(vf);
    w.w_v = A.template alloc<T>(vh);
  };
  if (p->precision == ICON_PREC_FP64) {
    build_ctx(en.c64, double{});
    // the FP64 stencils use the grid's own FP64 factors
    en.c64.g = en.g64;
  } else {
    build_ctx(en.c32, float{});
    if (!z_cols && p->fused_advection) {
      // rows A1-A4 of the FP32 stencils in one launch over patches of 128 cells
      HostVaPatches hp;
      const std::string err = build_va_patches(h, 128, &hp);
      if (!err.empty()) {
        A.release();
        delete d;
        return fail(ICON_ERR_ARG, fname + ": " + err);
      }
      // the grid factors the kernel reads, in patch order, rounded to FP32 as
      // the context's own factors are
      std::vector<float> e1_w(5 * hp.e1_g.size()), c3_w(4 * hp.c0_g.size(), 0.0f),
          v3_w(12 * hp.v3_g.size()), e4_w(4 * hp.e4_g.size(), 0.0f), own_w(4 * (size_t)nc, 0.0f);
      for (size_t i = 0; i < hp.e1_g.size(); ++i)
        for (int j = 0; j < 5; ++j) e1_w[5 * i + j] = (float)h.vt_w[5 * (size_t)hp.e1_g[i] + j];
      for (int q = 0; q < hp.n_patches; ++q)
        for (int i = 0; i < hp.n_c3[q]; ++i) {
          const size_t r = (size_t)hp.off_c0[q] + i;
          for (int j = 0; j < 3; ++j) c3_w[4 * r + j] = (float)h.e2c_w[3 * (size_t)hp.c0_g[r] + j];
        }
      for (size_t i = 0; i < hp.v3_g.size(); ++i)
        for (int j = 0; j < 6; ++j) {
          v3_w[12 * i + j] = (float)h.curl_v[6 * (size_t)hp.v3_g[i] + j];
          v3_w[12 * i + 6 + j] = (float)h.c2v_w[6 * (size_t)hp.v3_g[i] + j];
        }
      for (size_t i = 0; i < hp.e4_g.size(); ++i) {
        const int e = hp.e4_g[i];
        e4_w[4 * i] = (float)fe[e];
        e4_w[4 * i + 1] = (float)hinv_d[e];
        e4_w[4 * i + 2] = (float)d_o_l[e];
      }
      for (int c = 0; c < nc; ++c)
        for (int j = 0; j < 3; ++j) own_w[4 * (size_t)c + j] = (float)e2c_wd[3 * (size_t)c + j];
      VaPatchT& vp = en.c32.vp;
      vp.P = hp.P;
      vp.n_patches = hp.n_patches;
      vp.max_e0 = hp.max_e0;
      vp.max_e1 = hp.max_e1;
      vp.max_c3 = hp.max_c3;
      vp.max_c0 = hp.max_c0;
      vp.max_v3 = hp.max_v3;
      vp.max_e4 = hp.max_e4;
      vp.off_e0 = A.upload(hp.off_e0);
      vp.off_e1 = A.upload(hp.off_e1);
      vp.off_c0 = A.upload(hp.off_c0);
      vp.off_v3 = A.upload(hp.off_v3);
      vp.off_e4 = A.upload(hp.off_e4);
      vp.n_c3 = A.upload(hp.n_c3);
      vp.n_w4 = A.upload(hp.n_w4);
      vp.e0_g = A.upload(hp.e0_g);
      vp.c0_g = A.upload(hp.c0_g);
      vp.e4_g = A.upload(hp.e4_g);
      vp.e1_i = A.upload(hp.e1_i);
      vp.c3_i = A.upload(hp.c3_i);
      vp.v3_i = A.upload(hp.v3_i);
      vp.e4_i = A.upload(hp.e4_i);
      vp.own_i = A.upload(hp.own_i);
      vp.e1_w = A.upload(e1_w);
      vp.c3_w = A.upload(c3_w);
      vp.v3_w = A.upload(v3_w);
      vp.e4_w = A.upload(e4_w);
      vp.own_w = A.upload(own_w);
    }
    Mirrors& m = en.m;
    m.vn = A.alloc<float>(ef);
    m.w = A.alloc<float>(ch);
    m.rho = A.alloc<float>(cf);
    m.th = A.alloc<float>(cf);
    m.w_p = A.alloc<float>(ch);
  }

  // terrain: per-column reference state and column-solve table, and the
  // stencils' per-point metrics in their compute type
  if (z_cols) {
    en.terrain = true;
    v.exner_ref_c = A.upload(ht.exner_ref_c);
    v.theta_ref_c = A.upload(ht.theta_ref_c);
    v.dz_c = A.upload(ht.dz_c);
    if (p->precision == ICON_PREC_MIXED) {  // the double-word solve reads pairs
      std::vector<float> pairs(2 * ht.colt.size());
      for (size_t i = 0; i < ht.colt.size(); ++i) split_hl(ht.colt[i], &pairs[2 * i]);
      v.colt = reinterpret_cast<const double*>(A.upload(pairs));
    } else {
      v.colt = A.upload(ht.colt);
    }
    auto build_terr = [&](auto& x, auto tag) {
      using T = decltype(tag);
      auto up = [&](const std::vector<double>& src) { return A.upload(std::vector<T>(src.begin(), src.end())); };
      TerrT<T>& t = x.tr;
      t.wgt_e = up(ht.wgt_e);
      std::vector<double> q(ht.inv_dz_e);
      for (double& x : q) x *= 0.25;
      t.qdz_e = up(q);
      t.ddxn_ifc = up(ht.ddxn_ifc);
      t.ddxt_ifc = up(ht.ddxt_ifc);
      std::vector<double> cpd_ddxn(ht.ddxn_mc);
      for (double& x : cpd_ddxn) x *= p->cpd;
      t.ddxn_mc = up(cpd_ddxn);
      std::vector<double> qh(ht.inv_dzh_c);
      for (double& x : qh) x *= 0.5;
      t.qdzh_c = up(qh);
      t.inv_dzm_c = up(ht.inv_dzm_c);
      t.fx_ratio = up(ht.fx_ratio);
      t.wcc0 = A.template alloc<T>(ch);
      t.wcc1 = A.template alloc<T>(ch);
    };
    if (p->precision == ICON_PREC_FP64)
      build_terr(en.c64, double{});
    else
      build_terr(en.c32, float{});
    std::vector<double>().swap(ht.colt);  // the largest host copy, released early
    v.n_ray = std::max(v.n_ray, ht.n_ray);
    v.n_steep = (int)(ht.steep_w.size() / 6);
    if (v.n_steep > 0) {
      v.steep_idx = A.upload(ht.steep_idx);
      v.steep_w = A.upload(ht.steep_w);
    }
  }

  // FP64 work of the column solve and the predicted state
  DevWork& w = en.wk;
  w.div_m = A.alloc<double>(cf);
  w.div_t = A.alloc<double>(cf);
  w.rho_p = A.alloc<double>(cf);
  w.theta_p = A.alloc<double>(cf);
  w.w_p = A.alloc<double>(ch);
  w.pex = A.alloc<double>(cf);
  w.col = A.alloc<double>(7 * ch);
  w.zbl = A.alloc<double>(ch);
  w.diag = A.alloc<double>(diag_partials(nc));
  w.flag = A.alloc<int>(1);
  if (A.status == cudaSuccess) {
    cudaError_t e = cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) A.status = e;
  }
  if (A.status == cudaSuccess) {
    cudaError_t e = init_column_kernels();
    if (e == cudaSuccess && z_cols) e = init_column_terrain_kernels();
    if (e == cudaSuccess && en.c32.vp.n_patches > 0) e = init_va_fused(en.c32.vp);
    if (e != cudaSuccess) A.status = e;
  }
  if (A.status != cudaSuccess) {
    std::string m = fname + ": " + cudaGetErrorString(A.status);
    A.release();
    release_streams(d);
    delete d;
    return fail(ICON_ERR_CUDA, m);
  }
  {
    const bool mixed = is_mixed(p->precision);
    const DevVert& vv = en.v;
    const bool vert_ok = vv.dz && vv.inv_dz && vv.inv_dzh && vv.wgt && vv.theta_ref && vv.exner_ref &&
                         vv.dexner_ref_ic && vv.ray_fac && vv.colc && vv.lev_hl && vv.lev64;
    const bool terr_ok = !z_cols || (vv.exner_ref_c && vv.theta_ref_c && vv.dz_c && vv.colt &&
                                     (mixed ? terrain_complete(en.c32.tr) : terrain_complete(en.c64.tr)));
    const bool ok = vert_ok && terr_ok && grid_complete(en.g64) && work_complete(en.wk) &&
                    (mixed ? grid_complete(en.c32.g) : grid_complete(en.c64.g));
    if (!ok) {
      A.release();
      release_streams(d);
      delete d;
      return fail(ICON_ERR_CUDA, fname + ": internal error: a coefficient or work array is missing");
    }
  }
  for (int k = 0; k < kNumStencils; ++k) en.threads[k] = 256;
  en.col_kc = 4;
  if (p->autotune) {
    int rc = autotune(d);
    if (rc != ICON_OK) {
      A.release();
      release_streams(d);
      delete d;
      return rc;
    }
  }
  if (p->column_chunk) en.col_kc = p->column_chunk;
  *out = d;
  return ICON_OK;
}

}  // namespace

extern "C" {

int icon_dycore_destroy(icon_dycore_t* d) {
  if (!d) return ICON_OK;
  cudaStreamSynchronize(d->stream);
  free_graphs(d);
  if (d->io_stream) {
    cudaStreamSynchronize(d->io_stream);
    cudaStreamDestroy(d->io_stream);
    cudaEventDestroy(d->io_start);
    cudaEventDestroy(d->io_in);
    cudaEventDestroy(d->io_out);
  }
  if (d->have_staging) {
    cudaFree(d->staging.vn);
    cudaFree(d->staging.w);
    cudaFree(d->staging.rho);
    cudaFree(d->staging.exner);
    cudaFree(d->staging.theta_v);
    cudaFree(d->staging.exner_pr);
  }
  if (d->colx) {
    cudaFree(d->saved.vn);
    cudaFree(d->saved.w);
    cudaFree(d->saved.rho);
    cudaFree(d->saved.exner);
    cudaFree(d->saved.theta_v);
    cudaFree(d->saved.exner_pr);
    cudaFree(d->colx);
    cudaFree(d->status);
  }
  if (d->col16) cudaFree(d->col16);
  if (d->edge16) cudaFree(d->edge16);
  if (d->partial) cudaFree(d->partial);
  d->arena.release();
  release_streams(d);
  delete d;
  return ICON_OK;
}

}  // extern "C"

namespace {

enum class Where { kDevice, kHost, kMixed };

Where locate(const icon_state_t* s) {
  const void* ptrs[6] = {s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr};
  int ndev = 0;
  for (const void* p : ptrs) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;  // unknown to CUDA: plain host memory
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ++ndev;
  }
  if (ndev == 6) return Where::kDevice;
  if (ndev == 0) return Where::kHost;
  return Where::kMixed;
}

enum class Op { kStep, kSubstep, kDiffusion };

// io (whole steps of host arrays only): the step waits on d->io_in before
// it reads rho, theta_v, exner or exner_pr (after the first predictor's
// velocity tendencies in FP64; before the mirrors are refreshed in the mixed
// modes) and records d->io_out once rho and exner_pr are final (after the
// last corrector; the diffusion changes neither).
void enqueue(icon_dycore* d, Op op, const StateView& st, cudaStream_t s, bool io = false) {
  if (op == Op::kStep || op == Op::kSubstep) {
    int n = op == Op::kStep ? d->params.ndyn_substeps : 1;
    const bool mixed = is_mixed(d->en.precision);
    if (io && mixed) stream_wait_io(s, d->io_in);
    if (mixed) launch_refresh_mirrors(d->en, st, s);
    for (int i = 0; i < n; ++i) {
      d->en.io_wait = io && !mixed && i == 0 ? d->io_in : nullptr;
      if (mixed)
        launch_substep<float>(d->en, d->en.c32, st, s);
      else
        launch_substep<double>(d->en, d->en.c64, st, s);
      d->en.io_wait = nullptr;
    }
    if (io) stream_record_io(s, d->io_out);
  }
  if (op == Op::kStep || op == Op::kDiffusion) {
    if (is_mixed(d->en.precision)) {
      if (op == Op::kDiffusion) launch_refresh_mirrors(d->en, st, s);
      launch_diffusion<float>(d->en, d->en.c32, st, s);
    } else {
      launch_diffusion<double>(d->en, d->en.c64, st, s);
    }
  }
}

void enqueue_op(icon_dycore* d, int op, const StateView& st, cudaStream_t s) {
  enqueue(d, op == 0 ? Op::kStep : op == 1 ? Op::kSubstep : Op::kDiffusion, st, s);
}

thread_local Prof* g_user_prof = nullptr;

// per-kernel launch counts and summed event times of a finished profile
int summarise(const Prof& prof, int max_kernels, char* names, int32_t* launches, double* ms, int32_t* n_kernels,
              const char* fn) {
  std::vector<std::string> nm;
  std::vector<int> cnt;
  std::vector<double> tot;
  for (const auto& r : prof.recs) {
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, r.e0, r.e1));
    size_t j = 0;
    while (j < nm.size() && nm[j] != r.name) ++j;
    if (j == nm.size()) {
      nm.push_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[j] += 1;
    tot[j] += t;
  }
  if ((int)nm.size() > max_kernels) return fail(ICON_ERR_ARG, std::string(fn) + ": max_kernels too small");
  for (size_t j = 0; j < nm.size(); ++j) {
    std::snprintf(names + 64 * j, 64, "%s", nm[j].c_str());
    launches[j] = cnt[j];
    ms[j] = tot[j];
  }
  *n_kernels = (int32_t)nm.size();
  return ICON_OK;
}

bool same_state(const StateView& a, const StateView& b) {
  return a.vn == b.vn && a.w == b.w && a.rho == b.rho && a.exner == b.exner && a.theta_v == b.theta_v &&
         a.exner_pr == b.exner_pr;
}

// Graph of one full step for this set of state pointers; a cache of two
// entries covers double-buffered callers (as the paper's descriptor cache).
int step_graph(icon_dycore* d, const StateView& st, bool io, cudaGraphExec_t* exec) {
  ++d->use_counter;
  for (auto& e : d->graphs)
    if (e.exec && same_state(e.key, st) && e.io == io) {
      e.last_use = d->use_counter;
      *exec = e.exec;
      return ICON_OK;
    }
  GraphEntry* slot = &d->graphs[0];
  for (auto& e : d->graphs)
    if (!e.exec || e.last_use < slot->last_use) slot = &e;
  if (slot->exec) {
    CUDA_TRY(cudaStreamSynchronize(d->stream));
    cudaGraphExecDestroy(slot->exec);
    *slot = GraphEntry{};
  }
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal));
  enqueue(d, Op::kStep, st, d->cap_stream, io);
  cudaError_t le = cudaGetLastError();
  cudaError_t ee = cudaStreamEndCapture(d->cap_stream, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ICON_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(le));
  }
  CUDA_TRY(ee);
  cudaError_t ie = cudaGraphInstantiate(&slot->exec, graph, 0);
  cudaGraphDestroy(graph);
  CUDA_TRY(ie);
  slot->key = st;
  slot->io = io;
  slot->last_use = d->use_counter;
  *exec = slot->exec;
  return ICON_OK;
}

int run(icon_dycore* d, const icon_state_t* s, Op op, const char* name) {
  if (!d || !s) return fail(ICON_ERR_ARG, std::string(name) + ": NULL argument");
  if (!s->vn || !s->w || !s->rho || !s->exner || !s->theta_v || !s->exner_pr)
    return fail(ICON_ERR_ARG, std::string(name) + ": NULL state field");
  const HostGrid& h = d->grid->host;
  const int nlev = d->nlev;
  const size_t ef = (size_t)h.ne * nlev, cf = (size_t)h.nc * nlev, ch = (size_t)h.nc * (nlev + 1);
  Where where = locate(s);
  if (where == Where::kMixed)
    return fail(ICON_ERR_ARG, std::string(name) + ": state mixes host and device pointers");
  StateView st{s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr};
  cudaStream_t stream = d->stream;
  // a whole step of host arrays overlaps the copies of rho, exner, theta_v
  // and exner_pr with the first velocity tendencies and the copies of rho and
  // exner_pr back with the diffusion (on a private stream, ordered by events)
  const bool io = where == Where::kHost && op == Op::kStep;
  if (where == Where::kHost) {
    if (!d->have_staging) {
      StateView& g = d->staging;
      CUDA_TRY(cudaMalloc(&g.vn, ef * 8));
      CUDA_TRY(cudaMalloc(&g.w, ch * 8));
      CUDA_TRY(cudaMalloc(&g.rho, cf * 8));
      CUDA_TRY(cudaMalloc(&g.exner, cf * 8));
      CUDA_TRY(cudaMalloc(&g.theta_v, cf * 8));
      CUDA_TRY(cudaMalloc(&g.exner_pr, cf * 8));
      d->have_staging = true;
    }
    if (io && !d->io_stream) {  // all four or none
      cudaStream_t cs = nullptr;
      cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) {
        for (cudaEvent_t x : ev)
          if (x) cudaEventDestroy(x);
        if (cs) cudaStreamDestroy(cs);
        return fail(ICON_ERR_CUDA, std::string(name) + ": copy stream: " + cudaGetErrorString(e));
      }
      d->io_stream = cs;
      d->io_start = ev[0];
      d->io_in = ev[1];
      d->io_out = ev[2];
    }
    const StateView& g = d->staging;
    CUDA_TRY(cudaMemcpyAsync(g.vn, s->vn, ef * 8, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(g.w, s->w, ch * 8, cudaMemcpyHostToDevice, stream));
    // the other fields on the copy stream, after whatever the caller's stream holds
    cudaStream_t cs = io ? d->io_stream : stream;
    if (io) {
      CUDA_TRY(cudaEventRecord(d->io_start, stream));
      CUDA_TRY(cudaStreamWaitEvent(cs, d->io_start, 0));
    }
    CUDA_TRY(cudaMemcpyAsync(g.rho, s->rho, cf * 8, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(g.exner, s->exner, cf * 8, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(g.theta_v, s->theta_v, cf * 8, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(g.exner_pr, s->exner_pr, cf * 8, cudaMemcpyHostToDevice, cs));
    if (io) CUDA_TRY(cudaEventRecord(d->io_in, cs));
    st = g;
  }
  if (op == Op::kStep && d->params.use_graph && !g_prof) {
    cudaGraphExec_t exec = nullptr;
    int rc = step_graph(d, st, io, &exec);
    if (rc != ICON_OK) return rc;
    CUDA_TRY(cudaGraphLaunch(exec, stream));
  } else {
    enqueue(d, op, st, stream, io);
    CUDA_TRY(cudaGetLastError());
  }
  if (where == Where::kHost) {
    const StateView& g = d->staging;
    cudaStream_t cs = io ? d->io_stream : stream;
    if (io) CUDA_TRY(cudaStreamWaitEvent(cs, d->io_out, 0));
    CUDA_TRY(cudaMemcpyAsync(s->rho, g.rho, cf * 8, cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaMemcpyAsync(s->exner_pr, g.exner_pr, cf * 8, cudaMemcpyDeviceToHost, cs));
    CUDA_TRY(cudaMemcpyAsync(s->vn, g.vn, ef * 8, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(s->w, g.w, ch * 8, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(s->exner, g.exner, cf * 8, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(s->theta_v, g.theta_v, cf * 8, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (io) CUDA_TRY(cudaStreamSynchronize(cs));
  } else if (d->params.synchronous) {
    CUDA_TRY(cudaStreamSynchronize(stream));
  }
  return ICON_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint files of a state: a 64-byte header, then vn, w, rho, exner,
// theta_v and exner_pr as FP64 in the state's layout and the host's byte
// order (little-endian on the x86-64 and AArch64 hosts this library builds
// for).  The header carries a magic, a format version, the sizes and a
// checksum (FNV-1a over the payload's 64-bit words), so that a file of
// another grid or a damaged file is refused before the state is touched.
// ---------------------------------------------------------------------------
struct CheckpointHeader {
  char magic[8];
  uint32_t version, nlev;
  int64_t n_cells, n_edges;
  uint64_t payload_bytes, checksum;
  uint8_t reserved[16];
};
static_assert(sizeof(CheckpointHeader) == 64, "checkpoint header size");
constexpr char kCheckpointMagic[8] = {'I', 'C', 'O', 'N', 'D', 'Y', 'C', 'K'};
constexpr uint32_t kCheckpointVersion = 1;

uint64_t fnv1a_words(uint64_t h, const double* p, size_t n) {
  uint64_t w;
  for (size_t i = 0; i < n; ++i) {
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

struct FieldRef {
  double* p;
  size_t n;
};

int checkpoint_fields(icon_dycore* d, const icon_state_t* s, const char* fn, FieldRef (&f)[6], bool& device) {
  if (!d || !s) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL argument");
  if (!s->vn || !s->w || !s->rho || !s->exner || !s->theta_v || !s->exner_pr)
    return fail(ICON_ERR_ARG, std::string(fn) + ": NULL state field");
  const HostGrid& h = d->grid->host;
  const size_t ef = (size_t)h.ne * d->nlev, cf = (size_t)h.nc * d->nlev, ch = (size_t)h.nc * (d->nlev + 1);
  const Where where = locate(s);
  if (where == Where::kMixed) return fail(ICON_ERR_ARG, std::string(fn) + ": state mixes host and device pointers");
  device = where == Where::kDevice;
  f[0] = {s->vn, ef};
  f[1] = {s->w, ch};
  f[2] = {s->rho, cf};
  f[3] = {s->exner, cf};
  f[4] = {s->theta_v, cf};
  f[5] = {s->exner_pr, cf};
  return ICON_OK;
}

int checkpoint_save(icon_dycore* d, const icon_state_t* s, const char* path) {
  const char* fn = "icon_dycore_save";
  FieldRef f[6];
  bool device = false;
  int rc = checkpoint_fields(d, s, fn, f, device);
  if (rc != ICON_OK) return rc;
  if (!path) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL path");
  CUDA_TRY(cudaStreamSynchronize(d->stream));  // the state as the last enqueued step left it
  CheckpointHeader hd{};
  std::memcpy(hd.magic, kCheckpointMagic, 8);
  hd.version = kCheckpointVersion;
  hd.nlev = (uint32_t)d->nlev;
  hd.n_cells = d->grid->host.nc;
  hd.n_edges = d->grid->host.ne;
  for (const FieldRef& x : f) hd.payload_bytes += x.n * 8;
  hd.checksum = 0xcbf29ce484222325ull;
  FILE* out = std::fopen(path, "wb");
  if (!out) return fail(ICON_ERR_ARG, std::string(fn) + ": cannot open " + path + " for writing");
  bool ok = std::fwrite(&hd, sizeof hd, 1, out) == 1;
  std::vector<double> buf;
  for (int i = 0; i < 6 && ok; ++i) {
    const double* src = f[i].p;
    if (device) {
      buf.resize(f[i].n);
      const cudaError_t e = cudaMemcpy(buf.data(), f[i].p, f[i].n * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        std::fclose(out);
        return fail(ICON_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(e));
      }
      src = buf.data();
    }
    hd.checksum = fnv1a_words(hd.checksum, src, f[i].n);
    ok = std::fwrite(src, 8, f[i].n, out) == f[i].n;
  }
  ok = ok && std::fseek(out, 0, SEEK_SET) == 0 && std::fwrite(&hd, sizeof hd, 1, out) == 1;
  ok = (std::fclose(out) == 0) && ok;
  if (!ok) return fail(ICON_ERR_ARG, std::string(fn) + ": writing " + path + " failed");
  return ICON_OK;
}

int checkpoint_load(icon_dycore* d, const icon_state_t* s, const char* path) {
  const char* fn = "icon_dycore_load";
  FieldRef f[6];
  bool device = false;
  int rc = checkpoint_fields(d, s, fn, f, device);
  if (rc != ICON_OK) return rc;
  if (!path) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL path");
  FILE* in = std::fopen(path, "rb");
  if (!in) return fail(ICON_ERR_ARG, std::string(fn) + ": cannot open " + path);
  CheckpointHeader hd{};
  size_t payload = 0;
  for (const FieldRef& x : f) payload += x.n * 8;
  std::string why;
  if (std::fread(&hd, sizeof hd, 1, in) != 1) why = "no header";
  else if (std::memcmp(hd.magic, kCheckpointMagic, 8) != 0) why = "not a dycore checkpoint";
  else if (hd.version != kCheckpointVersion) why = "format version " + std::to_string(hd.version);
  else if (hd.nlev != (uint32_t)d->nlev || hd.n_cells != d->grid->host.nc || hd.n_edges != d->grid->host.ne ||
           hd.payload_bytes != payload)
    why = "sizes differ from this dycore's";
  std::vector<double> buf;
  // first pass: the checksum over the whole payload, before the state is touched
  uint64_t sum = 0xcbf29ce484222325ull;
  for (int i = 0; i < 6 && why.empty(); ++i) {
    buf.resize(f[i].n);
    if (std::fread(buf.data(), 8, f[i].n, in) != f[i].n) why = "file truncated";
    else sum = fnv1a_words(sum, buf.data(), f[i].n);
  }
  if (why.empty() && sum != hd.checksum) why = "checksum mismatch";
  // second pass: into the state
  if (why.empty() && std::fseek(in, (long)sizeof hd, SEEK_SET) != 0) why = "cannot rewind";
  if (why.empty()) {
    const cudaError_t e0 = cudaStreamSynchronize(d->stream);
    if (e0 != cudaSuccess) {
      std::fclose(in);
      return fail(ICON_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(e0));
    }
  }
  for (int i = 0; i < 6 && why.empty(); ++i) {
    double* dst = device ? nullptr : f[i].p;
    if (device) buf.resize(f[i].n);
    if (std::fread(device ? buf.data() : dst, 8, f[i].n, in) != f[i].n) {
      why = "file changed while reading";
      break;
    }
    if (device) {
      const cudaError_t e = cudaMemcpy(f[i].p, buf.data(), f[i].n * 8, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        std::fclose(in);
        return fail(ICON_ERR_CUDA, std::string(fn) + ": " + cudaGetErrorString(e));
      }
    }
  }
  std::fclose(in);
  if (!why.empty()) return fail(ICON_ERR_ARG, std::string(fn) + ": " + path + ": " + why);
  return ICON_OK;
}

}  // namespace

extern "C" {

int icon_dycore_step(icon_dycore_t* d, const icon_state_t* s) { return run(d, s, Op::kStep, "icon_dycore_step"); }
int icon_nh_solve(icon_dycore_t* d, const icon_state_t* s) { return run(d, s, Op::kSubstep, "icon_nh_solve"); }
int icon_nh_diff(icon_dycore_t* d, const icon_state_t* s) { return run(d, s, Op::kDiffusion, "icon_nh_diff"); }

int icon_velocity_tendencies(icon_dycore_t* d, const double* vn, const double* w, double* ddt_vn, double* ddt_w) {
  if (!d || !vn || !w || !ddt_vn || !ddt_w) return fail(ICON_ERR_ARG, "icon_velocity_tendencies: NULL argument");
  if (d->en.precision != ICON_PREC_FP64)
    return fail(ICON_ERR_UNSUPPORTED, "icon_velocity_tendencies: stage output is provided in FP64 mode only");
  launch_velocity_tendencies<double>(d->en.c64, vn, w, ddt_vn, ddt_w, nullptr, nullptr, d->stream, d->en.threads,
                                     d->en.terrain ? d->en.c64.tr.wcc0 : nullptr, d->en.shape);
  CUDA_TRY(cudaGetLastError());
  if (d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return ICON_OK;
}

int icon_dycore_reference_columns(const icon_dycore_t* d, double* theta_ref, double* exner_ref) {
  if (!d || !theta_ref || !exner_ref) return fail(ICON_ERR_ARG, "icon_dycore_reference_columns: NULL argument");
  const size_t nc = d->grid->host.nc, nlev = d->nlev;
  if (d->en.terrain) {
    CUDA_TRY(cudaMemcpy(theta_ref, d->en.v.theta_ref_c, nc * nlev * sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(exner_ref, d->en.v.exner_ref_c, nc * nlev * sizeof(double), cudaMemcpyDeviceToHost));
    return ICON_OK;
  }
  for (size_t c = 0; c < nc; ++c) {
    std::memcpy(theta_ref + c * nlev, d->theta_ref.data(), nlev * sizeof(double));
    std::memcpy(exner_ref + c * nlev, d->exner_ref.data(), nlev * sizeof(double));
  }
  return ICON_OK;
}

int icon_dycore_reference_state(const icon_dycore_t* d, double* theta_ref, double* exner_ref) {
  if (!d || !theta_ref || !exner_ref) return fail(ICON_ERR_ARG, "icon_dycore_reference_state: NULL argument");
  if (d->en.terrain)
    return fail(ICON_ERR_UNSUPPORTED,
                "icon_dycore_reference_state: the reference state varies by column over terrain; use "
                "icon_dycore_reference_columns");
  std::memcpy(theta_ref, d->theta_ref.data(), d->nlev * sizeof(double));
  std::memcpy(exner_ref, d->exner_ref.data(), d->nlev * sizeof(double));
  return ICON_OK;
}

int icon_dycore_profile(icon_dycore_t* d, const icon_state_t* s, int32_t nsteps, int32_t max_kernels, char* names,
                        int32_t* launches, double* ms, int32_t* n_kernels) {
  if (!d || !s || !names || !launches || !ms || !n_kernels || nsteps < 1 || max_kernels < 1)
    return fail(ICON_ERR_ARG, "icon_dycore_profile: NULL or invalid argument");
  if (!s->vn || !s->w || !s->rho || !s->exner || !s->theta_v || !s->exner_pr)
    return fail(ICON_ERR_ARG, "icon_dycore_profile: NULL state field");
  if (locate(s) != Where::kDevice) return fail(ICON_ERR_ARG, "icon_dycore_profile: state must be on the device");
  StateView st{s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr};
  Prof prof;
  g_prof = &prof;
  for (int i = 0; i < nsteps; ++i) enqueue(d, Op::kStep, st, d->stream);
  g_prof = nullptr;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return summarise(prof, max_kernels, names, launches, ms, n_kernels, "icon_dycore_profile");
}

int icon_profile_begin(void) {
  if (g_user_prof) return fail(ICON_ERR_ARG, "icon_profile_begin: a profile is already open on this thread");
  g_user_prof = new (std::nothrow) Prof();
  if (!g_user_prof) return fail(ICON_ERR_CUDA, "icon_profile_begin: out of memory");
  g_prof = g_user_prof;
  return ICON_OK;
}

int icon_profile_end(int32_t max_kernels, char* names, int32_t* launches, double* ms, int32_t* n_kernels) {
  if (!g_user_prof) return fail(ICON_ERR_ARG, "icon_profile_end: no profile open on this thread");
  g_prof = nullptr;
  Prof* prof = g_user_prof;
  g_user_prof = nullptr;
  int rc = ICON_OK;
  if (!names || !launches || !ms || !n_kernels) rc = fail(ICON_ERR_ARG, "icon_profile_end: NULL argument");
  if (rc == ICON_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = fail(ICON_ERR_CUDA, std::string("icon_profile_end: ") + cudaGetErrorString(e));
  }
  if (rc == ICON_OK) rc = summarise(*prof, max_kernels, names, launches, ms, n_kernels, "icon_profile_end");
  delete prof;
  return rc;
}

int icon_dycore_debug_field(icon_dycore_t* d, const char* name, void* dst, int64_t bytes) {
  if (!d || !name || !dst) return fail(ICON_ERR_ARG, "icon_dycore_debug_field: NULL argument");
  const HostGrid& h = d->grid->host;
  const size_t nlev = d->nlev, ef = h.ne * nlev, cf = h.nc * nlev, ch = h.nc * (nlev + 1);
  const bool mixed = is_mixed(d->en.precision);
  const size_t es = mixed ? sizeof(float) : sizeof(double);
  const void* src = nullptr;
  size_t n = 0;
  auto pick = [&](const char* nm, const void* p64, const void* p32, size_t count, size_t elem) {
    if (std::strcmp(name, nm) == 0) {
      src = mixed ? p32 : p64;
      n = count * elem;
    }
  };
  const WorkT<double>& a = d->en.c64.w;
  const WorkT<float>& b = d->en.c32.w;
  pick("vt", a.vt, b.vt, ef, es);
  pick("ekin_e", a.ekin_e, b.ekin_e, ef, es);
  pick("ddt_vn0", a.ddt_vn0, b.ddt_vn0, ef, es);
  pick("ddt_vn1", a.ddt_vn1, b.ddt_vn1, ef, es);
  pick("rho_e", a.rho_e, b.rho_e, ef, es);
  pick("theta_e", a.theta_e, b.theta_e, ef, es);
  pick("hpg", a.hpg, b.hpg, ef, es);
  pick("vn_p", a.vn_p, b.vn_p, ef, es);
  pick("divd", a.divd, b.divd, cf, es);
  pick("divd2", a.divd2, b.divd2, cf, es);
  pick("ddt_w0", a.ddt_w0, b.ddt_w0, ch, es);
  pick("ddt_w1", a.ddt_w1, b.ddt_w1, ch, es);
  pick("grad4", a.grad4, b.grad4, 4 * cf, es);
  pick("div_m", d->en.wk.div_m, d->en.wk.div_m, cf, sizeof(double));
  pick("div_t", d->en.wk.div_t, d->en.wk.div_t, cf, sizeof(double));
  pick("w_p", d->en.wk.w_p, d->en.m.w_p, ch, es);
  pick("rho_p", d->en.wk.rho_p, d->en.wk.rho_p, cf, sizeof(double));
  pick("theta_p", d->en.wk.theta_p, d->en.wk.theta_p, cf, sizeof(double));
  if (!src) return fail(ICON_ERR_ARG, std::string("icon_dycore_debug_field: unknown field ") + name);
  if (bytes < (int64_t)n) return fail(ICON_ERR_ARG, "icon_dycore_debug_field: destination too small");
  CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return ICON_OK;
}

int icon_dycore_diagnostics(icon_dycore_t* d, const icon_state_t* s, double* ps, double* t850, double* mass) {
  if (!d || !s) return fail(ICON_ERR_ARG, "icon_dycore_diagnostics: NULL argument");
  if (!s->vn || !s->w || !s->rho || !s->exner || !s->theta_v)
    return fail(ICON_ERR_ARG, "icon_dycore_diagnostics: NULL state field");
  const void* ptrs[5] = {s->vn, s->w, s->rho, s->exner, s->theta_v};
  for (const void* p : ptrs) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return fail(ICON_ERR_ARG, "icon_dycore_diagnostics: the state must be on the device");
    }
  }
  StateView st{s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr};
  const int nb = diag_partials(d->grid->host.nc);
  CUDA_TRY(cudaMemsetAsync(d->en.wk.flag, 0, sizeof(int), d->stream));
  launch_diagnostics(d->en, d->en.g64.cell_area, st, ps, t850, d->en.wk.diag, d->en.wk.flag, d->stream);
  CUDA_TRY(cudaGetLastError());
  std::vector<double> part(nb);
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(part.data(), d->en.wk.diag, nb * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaMemcpyAsync(&bad, d->en.wk.flag, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  if (mass) {
    double m = 0.0;
    for (double x : part) m += x;
    *mass = m;
  }
  if (bad) return fail(ICON_ERR_NUMERIC, "icon_dycore_diagnostics: the state holds non-finite values");
  return ICON_OK;
}

int icon_grid_cell_areas(const icon_grid_t* g, double* area) {
  if (!g || !area) return fail(ICON_ERR_ARG, "icon_grid_cell_areas: NULL argument");
  std::memcpy(area, g->host.cell_area.data(), g->host.nc * sizeof(double));
  return ICON_OK;
}

int icon_dycore_launch_config(const icon_dycore_t* d, char* buf, int32_t len) {
  if (!d || !buf || len < 1) return fail(ICON_ERR_ARG, "icon_dycore_launch_config: NULL or invalid argument");
  std::string s;
  for (int k = 0; k < kNumStencils; ++k) {
    s += kStencilNames[k];
    s += "=" + std::to_string(d->en.threads[k]);
    if (d->en.shape[k] >= 0) s += d->en.shape[k] ? "w" : "t";
    s += ",";
  }
  s += "column_threads=64;column_chunk=" + std::to_string(d->en.col_kc);
  std::snprintf(buf, (size_t)len, "%s", s.c_str());
  return ICON_OK;
}

int icon_dycore_synchronize(icon_dycore_t* d) {
  if (!d) return fail(ICON_ERR_ARG, "icon_dycore_synchronize: NULL argument");
  CUDA_TRY(cudaStreamSynchronize(d->stream));
  return ICON_OK;
}

int icon_dycore_sizes(const icon_dycore_t* d, int32_t* nlev, int32_t* nc, int32_t* ne, int32_t* nv) {
  if (!d) return fail(ICON_ERR_ARG, "icon_dycore_sizes: NULL argument");
  if (nlev) *nlev = d->nlev;
  if (nc) *nc = d->grid->host.nc;
  if (ne) *ne = d->grid->host.ne;
  if (nv) *nv = d->grid->host.nv;
  return ICON_OK;
}

int icon_dycore_save(icon_dycore_t* d, const icon_state_t* s, const char* path) {
  return checkpoint_save(d, s, path);
}

int icon_dycore_load(icon_dycore_t* d, const icon_state_t* s, const char* path) {
  return checkpoint_load(d, s, path);
}


}  // extern "C"

namespace {

bool on_device(const icon_state_t* s) {
  const void* ptrs[6] = {s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr};
  for (const void* p : ptrs) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

StateView view(const icon_state_t* s) { return StateView{s->vn, s->w, s->rho, s->exner, s->theta_v, s->exner_pr}; }

int learned_buffers(icon_dycore* d, int partials, int ldc, int lde) {
  const HostGrid& h = d->grid->host;
  const size_t nlev = d->nlev, ef = (size_t)h.ne * nlev, cf = (size_t)h.nc * nlev, ch = (size_t)h.nc * (nlev + 1);
  if (!d->colx) {
    StateView& g = d->saved;
    CUDA_TRY(cudaMalloc(&g.vn, ef * 8));
    CUDA_TRY(cudaMalloc(&g.w, ch * 8));
    CUDA_TRY(cudaMalloc(&g.rho, cf * 8));
    CUDA_TRY(cudaMalloc(&g.exner, cf * 8));
    CUDA_TRY(cudaMalloc(&g.theta_v, cf * 8));
    CUDA_TRY(cudaMalloc(&g.exner_pr, cf * 8));
    CUDA_TRY(cudaMalloc(&d->colx, cf * 5 * 4));
    CUDA_TRY(cudaMalloc(&d->status, (2 + (size_t)reduce_stage_doubles()) * sizeof(double)));
  }
  // BF16 network inputs; the pad columns stay zero (the kernels write only the features)
  if (ldc != d->ld_col16) {
    if (d->col16) cudaFree(d->col16);
    d->col16 = nullptr;
    CUDA_TRY(cudaMalloc(&d->col16, (size_t)h.nc * ldc * sizeof(__nv_bfloat16)));
    CUDA_TRY(cudaMemset(d->col16, 0, (size_t)h.nc * ldc * sizeof(__nv_bfloat16)));
    d->ld_col16 = ldc;
  }
  if (lde != d->ld_edge16) {
    if (d->edge16) cudaFree(d->edge16);
    d->edge16 = nullptr;
    CUDA_TRY(cudaMalloc(&d->edge16, (size_t)h.ne * lde * sizeof(__nv_bfloat16)));
    CUDA_TRY(cudaMemset(d->edge16, 0, (size_t)h.ne * lde * sizeof(__nv_bfloat16)));
    d->ld_edge16 = lde;
  }
  if (partials > d->partial_cap) {
    if (d->partial) cudaFree(d->partial);
    d->partial = nullptr;
    CUDA_TRY(cudaMalloc(&d->partial, (size_t)partials * sizeof(float)));
    d->partial_cap = partials;
  }
  return ICON_OK;
}

int copy_state(const StateView& dst, const StateView& src, const icon_dycore* d, cudaStream_t s) {
  const HostGrid& h = d->grid->host;
  const size_t nlev = d->nlev, ef = (size_t)h.ne * nlev, cf = (size_t)h.nc * nlev, ch = (size_t)h.nc * (nlev + 1);
  CUDA_TRY(cudaMemcpyAsync(dst.vn, src.vn, ef * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst.w, src.w, ch * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst.rho, src.rho, cf * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst.exner, src.exner, cf * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst.theta_v, src.theta_v, cf * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dst.exner_pr, src.exner_pr, cf * 8, cudaMemcpyDeviceToDevice, s));
  return ICON_OK;
}

// checks that a network maps n_in -> n_out and carries normalisation statistics
int check_net(const icon_mlp_t* net, int n_in, int n_out, const char* which) {
  int ni = 0, no = 0, mb = 0;
  mlp_dims(net, &ni, &no, &mb);
  if (ni != n_in || no != n_out)
    return fail(ICON_ERR_ARG, std::string("icon_dycore_step_learned: ") + which + " network must map " +
                                  std::to_string(n_in) + " -> " + std::to_string(n_out));
  const float *xm, *xs, *ym, *ys;
  mlp_norm(net, &xm, &xs, &ym, &ys);
  if (!xm) return fail(ICON_ERR_ARG, std::string("icon_dycore_step_learned: ") + which + " network has no normalisation");
  return ICON_OK;
}

}  // namespace

extern "C" {

int icon_corrector_features(icon_dycore_t* d, const icon_state_t* s, float* col_x, float* edge_x) {
  if (!d || !s || !col_x || !edge_x) return fail(ICON_ERR_ARG, "icon_corrector_features: NULL argument");
  if ((double)d->grid->host.ne * (11.0 * d->nlev) >= 4294967295.0)
    return fail(ICON_ERR_ARG, "icon_corrector_features: grid too large for 32-bit indexing");
  if (!on_device(s)) return fail(ICON_ERR_ARG, "icon_corrector_features: the state must be on the device");
  const StateView st = view(s);
  launch_col_features(d->en, st, col_x, nullptr, 0, nullptr, nullptr, d->stream);
  launch_edge_features(d->en, col_x, st.vn, edge_x, 11 * d->nlev, nullptr, nullptr, d->stream);
  CUDA_TRY(cudaGetLastError());
  if (d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return ICON_OK;
}

int icon_corrector_targets(icon_dycore_t* d, const icon_state_t* reduced, const icon_state_t* plain, float* col_y,
                           float* edge_y) {
  if (!d || !reduced || !plain || !col_y || !edge_y) return fail(ICON_ERR_ARG, "icon_corrector_targets: NULL argument");
  if ((double)d->grid->host.nc * (3.0 * d->nlev) >= 4294967295.0)
    return fail(ICON_ERR_ARG, "icon_corrector_targets: grid too large for 32-bit indexing");
  if (!on_device(reduced) || !on_device(plain))
    return fail(ICON_ERR_ARG, "icon_corrector_targets: the states must be on the device");
  launch_targets(d->en, view(reduced), view(plain), col_y, edge_y, d->stream);
  CUDA_TRY(cudaGetLastError());
  if (d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return ICON_OK;
}

int icon_dycore_step_learned(icon_dycore_t* reduced, icon_dycore_t* plain, icon_mlp_t* col_net, icon_mlp_t* edge_net,
                             const icon_state_t* s, double max_norm, int32_t* used_fallback, double* norm) {
  const char* fn = "icon_dycore_step_learned";
  if (!reduced || !plain || !col_net || !edge_net || !s) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL argument");
  if (reduced->grid != plain->grid || reduced->nlev != plain->nlev)
    return fail(ICON_ERR_ARG, std::string(fn) + ": the two dycores must share the grid and the levels");
  if (!on_device(s)) return fail(ICON_ERR_ARG, std::string(fn) + ": the state must be on the device");
  const HostGrid& h = reduced->grid->host;
  const int nlev = reduced->nlev, nc = h.nc, ne = h.ne;
  int rc = check_net(col_net, 5 * nlev, 3 * nlev - 1, "column");
  if (rc != ICON_OK) return rc;
  rc = check_net(edge_net, 11 * nlev, nlev, "edge");
  if (rc != ICON_OK) return rc;
  int ni, no, mbc, mbe;
  mlp_dims(col_net, &ni, &no, &mbc);
  mlp_dims(edge_net, &ni, &no, &mbe);
  // the feature and increment kernels index one chunk or one field with 32 bits
  if ((double)std::max(mbc, mbe) * (11.0 * nlev) >= 4294967295.0 || (double)ne * (11.0 * nlev) >= 4294967295.0)
    return fail(ICON_ERR_ARG, std::string(fn) + ": grid or network batch too large for 32-bit indexing");
  // partial-sum slots: one per 256 outputs of every chunk
  int pc = 0, pe = 0;
  for (int r0 = 0; r0 < nc; r0 += mbc) pc += apply_partials((size_t)std::min(mbc, nc - r0) * (3 * nlev - 1));
  for (int r0 = 0; r0 < ne; r0 += mbe) pe += apply_partials((size_t)std::min(mbe, ne - r0) * nlev);
  rc = learned_buffers(reduced, pc + pe, mlp_input_ld(col_net), mlp_input_ld(edge_net));
  if (rc != ICON_OK) return rc;
  icon_dycore* d = reduced;
  cudaStream_t stream = d->stream;
  const StateView st = view(s);
  // 1. keep the input state for the fallback; 2. the reduced step
  rc = copy_state(d->saved, st, d, stream);
  if (rc != ICON_OK) return rc;
  const int sync = d->params.synchronous;
  d->params.synchronous = 0;
  rc = run(d, s, Op::kStep, fn);
  d->params.synchronous = sync;
  if (rc != ICON_OK) return rc;
  // 3. features of the reduced state, normalised, as the networks' BF16 input rows
  const float *cxm, *cxi, *cym, *cys, *exm, *exi, *eym, *eys;
  mlp_norm(col_net, &cxm, &cxi, &cym, &cys);
  mlp_norm(edge_net, &exm, &exi, &eym, &eys);
  launch_col_inputs(d->en, st, d->colx, d->col16, d->ld_col16, cxm, cxi, stream);
  launch_edge_inputs(d->en, d->colx, st.vn, d->edge16, d->ld_edge16, exm, exi, stream);
  // 4. both networks over row chunks, increments applied as each chunk comes out
  int off = 0;
  for (int r0 = 0; r0 < nc; r0 += mbc) {
    const int rows = std::min(mbc, nc - r0);
    const float* y;
    int ldy;
    rc = mlp_forward_rows(col_net, d->col16 + (size_t)r0 * d->ld_col16, d->ld_col16, rows, &y, &ldy, stream);
    if (rc != ICON_OK) return rc;
    launch_apply_col(d->en, r0, rows, y, ldy, cym, cys, st, d->partial + off, stream);
    off += apply_partials((size_t)rows * (3 * nlev - 1));
  }
  for (int r0 = 0; r0 < ne; r0 += mbe) {
    const int rows = std::min(mbe, ne - r0);
    const float* y;
    int ldy;
    rc = mlp_forward_rows(edge_net, d->edge16 + (size_t)r0 * d->ld_edge16, d->ld_edge16, rows, &y, &ldy, stream);
    if (rc != ICON_OK) return rc;
    launch_apply_edge(d->en, r0, rows, y, ldy, eym, eys, st.vn, d->partial + off, stream);
    off += apply_partials((size_t)rows * nlev);
  }
  // 5. the check: RMS of the normalised increments of each network (NaN if anything is non-finite)
  launch_reduce_status(d->partial, pc, pe, d->status + 2, d->status, stream);
  CUDA_TRY(cudaGetLastError());
  double ss[2] = {0.0, 0.0};
  int tc_err = 0;
  const int* tc_flag = mlp_tc_error_flag();
  if (!tc_flag) return fail(ICON_ERR_CUDA, std::string(fn) + ": cannot read the GEMM status");
  CUDA_TRY(cudaMemcpyAsync(ss, d->status, sizeof(ss), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaMemcpyAsync(&tc_err, tc_flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (tc_err) return fail(ICON_ERR_CUDA, std::string(fn) + ": a tensor-core GEMM timed out waiting for its pipeline");
  const double rms = std::max(std::sqrt(ss[0] / ((double)nc * (3 * nlev - 1))), std::sqrt(ss[1] / ((double)ne * nlev)));
  const double r = std::isnan(ss[0] + ss[1]) ? NAN : rms;
  if (norm) *norm = r;
  const bool reject = !(r <= max_norm);
  if (used_fallback) *used_fallback = reject ? 1 : 0;
  if (reject) {
    // 6. fallback: the plain step from the saved input state
    rc = copy_state(st, d->saved, d, stream);
    if (rc != ICON_OK) return rc;
    if (plain->stream != stream) CUDA_TRY(cudaStreamSynchronize(stream));
    rc = run(plain, s, Op::kStep, fn);
    if (rc != ICON_OK) return rc;
    if (plain->stream != stream) CUDA_TRY(cudaStreamSynchronize(plain->stream));
  }
  if (d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(stream));
  return ICON_OK;
}

}  // extern "C"

namespace {

// Checks and runs the blocked <-> level-contiguous copy of all six fields.
int blocked_copy(icon_dycore* d, int nproma, const icon_state_t* from, const icon_state_t* to, bool to_blocked,
                 const char* fn) {
  if (!d || !from || !to) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL argument");
  if (!on_device(from) || !on_device(to)) return fail(ICON_ERR_ARG, std::string(fn) + ": states must be on the device");
  const HostGrid& h = d->grid->host;
  if (nproma < 1 || (h.ne + nproma - 1) / nproma > 65535 || (h.nc + nproma - 1) / nproma > 65535)
    return fail(ICON_ERR_ARG, std::string(fn) + ": nproma must be >= 1 with at most 65535 blocks");
  const StateView a = view(from), b = view(to);
  const double* fa[6] = {a.vn, a.w, a.rho, a.exner, a.theta_v, a.exner_pr};
  const double* fb[6] = {b.vn, b.w, b.rho, b.exner, b.theta_v, b.exner_pr};
  for (int f = 0; f < 6; ++f)
    for (int g = 0; g < 6; ++g)
      if (fa[f] == fb[g]) return fail(ICON_ERR_ARG, std::string(fn) + ": source and destination arrays overlap");
  const int nlev = d->nlev;
  launch_blocked(to_blocked, h.ne, nlev, nproma, a.vn, b.vn, d->stream);
  launch_blocked(to_blocked, h.nc, nlev + 1, nproma, a.w, b.w, d->stream);
  launch_blocked(to_blocked, h.nc, nlev, nproma, a.rho, b.rho, d->stream);
  launch_blocked(to_blocked, h.nc, nlev, nproma, a.exner, b.exner, d->stream);
  launch_blocked(to_blocked, h.nc, nlev, nproma, a.theta_v, b.theta_v, d->stream);
  launch_blocked(to_blocked, h.nc, nlev, nproma, a.exner_pr, b.exner_pr, d->stream);
  CUDA_TRY(cudaGetLastError());
  return ICON_OK;
}

}  // namespace

extern "C" {

int icon_state_from_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* blocked, const icon_state_t* state) {
  int rc = blocked_copy(d, nproma, blocked, state, false, "icon_state_from_blocked");
  if (rc == ICON_OK && d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return rc;
}

int icon_state_to_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* state, const icon_state_t* blocked) {
  int rc = blocked_copy(d, nproma, state, blocked, true, "icon_state_to_blocked");
  if (rc == ICON_OK && d->params.synchronous) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return rc;
}

int icon_dycore_step_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* blocked) {
  const char* fn = "icon_dycore_step_blocked";
  if (!d || !blocked) return fail(ICON_ERR_ARG, std::string(fn) + ": NULL argument");
  const HostGrid& h = d->grid->host;
  const size_t nlev = d->nlev, ef = (size_t)h.ne * nlev, cf = (size_t)h.nc * nlev, ch = (size_t)h.nc * (nlev + 1);
  if (!d->have_staging) {
    StateView& g = d->staging;
    CUDA_TRY(cudaMalloc(&g.vn, ef * 8));
    CUDA_TRY(cudaMalloc(&g.w, ch * 8));
    CUDA_TRY(cudaMalloc(&g.rho, cf * 8));
    CUDA_TRY(cudaMalloc(&g.exner, cf * 8));
    CUDA_TRY(cudaMalloc(&g.theta_v, cf * 8));
    CUDA_TRY(cudaMalloc(&g.exner_pr, cf * 8));
    d->have_staging = true;
  }
  const StateView& g = d->staging;
  const icon_state_t lib{g.vn, g.w, g.rho, g.exner, g.theta_v, g.exner_pr};
  int rc = blocked_copy(d, nproma, blocked, &lib, false, fn);
  if (rc != ICON_OK) return rc;
  const int sync = d->params.synchronous;
  d->params.synchronous = 0;
  rc = run(d, &lib, Op::kStep, fn);
  d->params.synchronous = sync;
  if (rc != ICON_OK) return rc;
  rc = blocked_copy(d, nproma, &lib, blocked, true, fn);
  if (rc == ICON_OK && sync) CUDA_TRY(cudaStreamSynchronize(d->stream));
  return rc;
}

}  // extern "C"

