/*
 * icon_dycore.h -- C-ABI of the GB300 ICON-type nonhydrostatic dynamical core.
 *
 * The paper (Sec. 4.3) plugs a dynamical core into the ICON Fortran model
 * through a C-ABI function: the host gathers pointers to the fields the
 * dynamics needs and passes them, scalars by value and arrays by reference
 * without copies, device arrays included (Sec. 4.3.1); setup-phase arrays
 * (connectivity, geometry) are passed once.  This header is that boundary for
 * a hand-written CUDA dycore: plain C types, no C++ or torch types, callable
 * from Fortran through iso_c_binding.
 *
 * The step it advances (Sec. 4.1, Fig. 1): ndyn_substeps dynamical substeps
 * (``nh_solve``, each a predictor and a corrector: velocity advection,
 * horizontal momentum update with pressure gradient and upwind rho/theta_v
 * fluxes, divergence damping in the corrector, vertically implicit solve for
 * w and the thermodynamic state) followed by one diffusion call (``nh_diff``,
 * Smagorinsky plus fourth-order background), Sec. 5.1.
 *
 * Conventions shared by every entry point
 *  - Return value: ICON_OK (0) on success, a negative ICON_ERR_* code on
 *    failure; icon_last_error() then returns a message (thread-local,
 *    valid until the next failing call on the same thread).  On failure
 *    no output is written unless stated otherwise.
 *  - Ownership: every array passed in stays owned by the caller.  The
 *    library copies what it keeps (grid tables, vertical grid) and owns its
 *    coefficient arrays, scratch and CUDA graphs, freed by *_destroy.
 *  - Field layout: level-contiguous, X[h * nlev_x + k], h the horizontal
 *    index (cell, edge or vertex), k the level; k = 0 is the model top.
 *    Full levels: nlev_x = nlev.  Half levels (w): nlev_x = nlev + 1, with
 *    k = nlev the ground.  This is the Fortran array X(nlev_x, n_h).
 *  - Index tables are int32 in the caller's index_base (0 for C, 1 for
 *    Fortran); "pad" entries of the 6-wide vertex tables equal
 *    index_base - 1 (pentagon vertices have 5 neighbours).
 *  - Logical flags are int32 (Fortran LOGICAL is 4 bytes; Sec. 4.3.1).
 */
#ifndef ICON_DYCORE_H
#define ICON_DYCORE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ICON_OK 0
#define ICON_ERR_ARG (-1)          /* NULL / out-of-range argument */
#define ICON_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define ICON_ERR_GRID (-3)         /* grid tables or coordinates inconsistent */
#define ICON_ERR_NUMERIC (-4)      /* non-finite or out-of-range state detected */
#define ICON_ERR_UNSUPPORTED (-5)  /* valid request the library does not implement */

#define ICON_PREC_FP64 0           /* every stencil and update in FP64 */
#define ICON_PREC_MIXED 1          /* FP32 stencils, double-word FP32 column solve, FP64 state updates */
#define ICON_PREC_MIXED_F64COL 2   /* FP32 stencils, FP64 column solve, FP64 state updates */

typedef struct icon_grid icon_grid_t;      /* opaque */
typedef struct icon_dycore icon_dycore_t;  /* opaque */

/*
 * Horizontal grid (Sec. 5.1: icosahedral RnBm triangular grid).
 * All pointers are HOST pointers, read during icon_grid_create only.
 *   c2v [n_cells*3]  cell vertices, counter-clockwise seen from outside
 *   c2e [n_cells*3]  cell edges
 *   e2c [n_edges*2]  the two cells of an edge; the edge normal points
 *                    from e2c[2e] to e2c[2e+1]  (sign convention of vn)
 *   e2v [n_edges*2]  the two vertices of an edge (any order)
 *   v2e [n_verts*6]  edges around a vertex, pad = index_base - 1
 *   v2c [n_verts*6]  cells around a vertex, pad = index_base - 1
 *   cell_xyz [n_cells*3]  cell circumcentres, unit vectors
 *   vert_xyz [n_verts*3]  vertices, unit vectors
 *   edge_xyz [n_edges*3]  edge (arc) midpoints, unit vectors
 * The library derives every geometric factor (areas, lengths, normals,
 * interpolation and reconstruction weights) from these.
 */
typedef struct icon_grid_desc {
  int32_t n_cells, n_edges, n_verts;
  int32_t index_base;
  double sphere_radius; /* m */
  const int32_t* c2v;
  const int32_t* c2e;
  const int32_t* e2c;
  const int32_t* e2v;
  const int32_t* v2e;
  const int32_t* v2c;
  const double* cell_xyz;
  const double* vert_xyz;
  const double* edge_xyz;
} icon_grid_desc_t;

/* Validate the tables (ranges, cell/edge/vertex consistency, unit vectors)
 * and build the grid (Sec. 5.1: the RnBm grid; Sec. 4.3: the host model hands
 * over its own tables, as ICON does with its grid).  Errors: ICON_ERR_ARG (NULL pointer, bad counts or
 * index_base), ICON_ERR_GRID (inconsistent tables), ICON_ERR_CUDA. */
int icon_grid_create(const icon_grid_desc_t* desc, icon_grid_t** out);
/* NULL-safe.  A grid must outlive every dycore created on it (Sec. 4.3: the
 * host model owns the lifetime of what it creates through the interface). */
int icon_grid_destroy(icon_grid_t* grid);

/*
 * Time-step and scheme parameters (Sec. 4.1 names the parts, not the
 * values; the defaults are ICON-like).  Fill with icon_dycore_params_default
 * and override.  Times in s, lengths in m.
 */
typedef struct icon_dycore_params {
  double dtime;            /* time step; the substep is dtime/ndyn_substeps */
  int32_t ndyn_substeps;   /* dynamical substeps per step (Sec. 4.1, 5.1) */
  /* physical constants */
  double grav, rd, cpd, p00, omega;
  /* solve_nonhydro */
  double vwind_impl_wgt;   /* implicit weight beta of the vertical solve, in (0, 1] */
  double wgt_nnow_vel, wgt_nnew_vel;  /* corrector weights of the advective tendencies */
  double wgt_nnow_rth, wgt_nnew_rth;  /* corrector weights of rho, theta_v */
  double exner_exfac;      /* exner-perturbation time extrapolation factor */
  double divdamp_fac;      /* fourth-order divergence damping (corrector only) */
  double divflux_fac;      /* mass-flux velocity filter vn + fac*Abar*grad_n(div vn); 0 = off */
  double rayleigh_coeff;   /* Rayleigh damping of w, 1/s; 0 = off */
  double damp_height;      /* Rayleigh damping acts above this height */
  /* diffusion */
  double hdiff_smag_fac;   /* Smagorinsky factor */
  double hdiff_k4;         /* fourth-order background coefficient of vn (x A_e^2) */
  double hdiff_w_k4;       /* fourth-order coefficient of w (x A_c^2) */
  int32_t hdiff_temp;      /* logical: diffuse theta_v and adjust exner */
  /* reference state theta_ref(z) = ref_T0 exp(z/H), H = cpd ref_T0 / grav */
  double ref_T0;
  /* execution */
  int32_t precision;       /* ICON_PREC_FP64, ICON_PREC_MIXED or ICON_PREC_MIXED_F64COL */
  int32_t use_graph;       /* logical: replay a captured CUDA graph per step */
  int32_t autotune;        /* logical: pick per-kernel launch shapes at create time */
  int32_t synchronous;     /* logical: return only after the GPU work ended */
  void* stream;            /* cudaStream_t to enqueue on; NULL = default stream */
  int32_t column_chunk;    /* levels per shared-memory chunk of the column solve: 4, 6 or 8;
                              0 = 4, or the autotuner's choice when autotune is set */
  /* steep terrain (Sec. 4.1: the dycore runs over real orography; its diffusion
   * raises the coefficients for strong near-surface temperature gradients) */
  int32_t steep_hpg;       /* logical, terrain only: the horizontal pressure gradient at
                              constant height (quadratic interpolation of the total exner
                              of each cell to the edge's height) at edge levels where the
                              two cells' levels are offset by more than half a layer */
  double hdiff_tenh_fac;   /* enhanced temperature diffusion: edge coefficient
                              fac A_e / dtime max(e_c0, e_c1); 0 = off */
  double hdiff_tenh_thresh;  /* K: e_c = min(1, (|theta_c - mean of its 3 neighbours| - thresh)/thresh) */
  int32_t hdiff_tenh_levels; /* the lowest levels where e_c may be nonzero
                                (>= 0; more than nlev means every level) */
  int32_t fused_advection;  /* logical (default 0), mixed precision over flat
                               ground: the velocity tendencies (rows A1-A4) in one
                               kernel over patches of 128 cells, intermediates in
                               shared memory; the same bits as the four separate
                               kernels, and on GB300 about 1.3x their time */
} icon_dycore_params_t;

/* Writes the defaults (Sec. 4.1 names the scheme's parts, not its values;
 * these are ICON-like): dtime 1800, ndyn_substeps 5, beta 0.65, tendency
 * weights 0.25/0.75, rho/theta weights 0.6/0.4, exner_exfac 1/3,
 * divdamp_fac 0.0025, divflux_fac 0.07, Rayleigh off (coeff 0, height 20 km), Smagorinsky
 * 0.015, k4 = k4w = 1/288, hdiff_temp 1, ref_T0 250, FP64, graph on,
 * autotune on, synchronous, default stream, steep_hpg off, enhanced
 * temperature diffusion off (factor 0, threshold 5 K, lowest 5 levels).
 * NULL-safe (does nothing). */
void icon_dycore_params_default(icon_dycore_params_t* p);

/*
 * Create a dycore on a grid with nlev flat height levels (Sec. 4.1: the
 * nonhydrostatic dynamical core; Sec. 4.3: created once at model set-up and
 * stepped from the time loop).
 *   z_ifc [nlev+1]: HOST pointer, half-level heights in m, top first,
 *                   strictly decreasing, z_ifc[nlev] = 0 (flat ground).
 * Derives the vertical metrics and the reference state, uploads all
 * coefficients, allocates scratch for one step.  The parameters are copied.
 * Errors: ICON_ERR_ARG, ICON_ERR_UNSUPPORTED (precision mode not built),
 * ICON_ERR_CUDA (e.g. out of device memory).
 */
int icon_dycore_create(const icon_grid_t* grid, int32_t nlev, const double* z_ifc,
                       const icon_dycore_params_t* params, icon_dycore_t** out);
/*
 * Create a dycore over terrain: a terrain-following height coordinate with
 * half-level heights per column (Sec. 4.1: ICON's dynamical core runs over
 * real orography; Sec. 5: the global configurations include topography).
 *   z_ifc [n_cells*(nlev+1)]: HOST pointer, level-contiguous like a w field,
 *          z_ifc[c*(nlev+1) + k] the height of half level k of column c in m;
 *          strictly decreasing in every column, the model top z_ifc[c*(nlev+1)]
 *          the same in every column (a flat top); the ground
 *          z_ifc[c*(nlev+1) + nlev] is the topography.
 * Per column: the vertical metrics, the reference state (discretely balanced
 * along the column) and the column solve's coefficients.  At edges: layer
 * thicknesses and interpolation weights from the mean of the two cells'
 * heights, and the slopes of the coordinate surfaces.  The step then uses the
 * contravariant vertical velocity w - w_concorr (w_concorr the vertical
 * velocity of a parcel following the coordinate surface) for vertical
 * advection and in the implicit solve, which keeps w = w_concorr at the
 * ground (kinematic condition); the horizontal pressure gradient is taken
 * along the true horizontal; horizontal fluxes carry the edge layer
 * thickness, so the total mass stays conserved.  Diffusion acts along the
 * coordinate surfaces.  With equal columns the step equals that of
 * icon_dycore_create on the same heights bit for bit.  exner_pr and the
 * diagnostics use the per-column reference state (icon_dycore_reference_columns).
 * Errors: as icon_dycore_create; ICON_ERR_ARG for heights that are not finite,
 * not decreasing or without a common top.
 */
int icon_dycore_create_terrain(const icon_grid_t* grid, int32_t nlev, const double* z_ifc,
                               const icon_dycore_params_t* params, icon_dycore_t** out);

/* NULL-safe; frees library-owned memory only (Sec. 4.3: the state arrays
 * stay the caller's). */
int icon_dycore_destroy(icon_dycore_t* dycore);

/*
 * Prognostic state, FP64, caller-owned, updated IN PLACE by the step calls.
 *   vn       [n_edges*nlev]      edge-normal wind, m/s
 *   w        [n_cells*(nlev+1)]  vertical wind at half levels, m/s
 *   rho      [n_cells*nlev]      density, kg/m^3
 *   exner    [n_cells*nlev]      Exner pressure
 *   theta_v  [n_cells*nlev]      virtual potential temperature, K
 *   exner_pr [n_cells*nlev]      exner - exner_ref of the previous substep
 *                                (extrapolation history; at a cold start
 *                                set it to exner - exner_ref, see
 *                                icon_dycore_reference_state)
 * Either all six are device pointers (no copies; the calls enqueue on the
 * dycore's stream), or all six are host pointers (the library copies in and
 * out around the call and returns when the copies back are done; pinned
 * memory copies fastest).  In a full step of host arrays, rho, exner,
 * theta_v and exner_pr are copied in on a second, library-owned stream while
 * the first velocity tendencies run, and rho and exner_pr back while the
 * diffusion runs; the results are those of a device-array step, bit for bit.
 */
typedef struct icon_state {
  double* vn;
  double* w;
  double* rho;
  double* exner;
  double* theta_v;
  double* exner_pr;
} icon_state_t;

/* One full time step: ndyn_substeps calls of the substep, then diffusion
 * (Sec. 4.1, Sec. 5.1), as one CUDA graph when params.use_graph is set.
 * Errors: ICON_ERR_ARG (NULL field, mixed host/device pointers),
 * ICON_ERR_CUDA. */
int icon_dycore_step(icon_dycore_t* dycore, const icon_state_t* state);

/* One dynamical substep, predictor + corrector, of length
 * dtime/ndyn_substeps: the paper's nh_solve (Sec. 4.1, 5.1). */
int icon_nh_solve(icon_dycore_t* dycore, const icon_state_t* state);

/* Horizontal diffusion over dtime: the paper's nh_diff (Sec. 4.1, 5.1). */
int icon_nh_diff(icon_dycore_t* dycore, const icon_state_t* state);

/* Advective tendencies alone (the first part of every predictor and
 * corrector, Sec. 4.1), for stage-level verification as in Sec. 4.4:
 *   vn [n_edges*nlev], w [n_cells*(nlev+1)]        inputs
 *   ddt_vn [n_edges*nlev], ddt_w [n_cells*(nlev+1)] outputs
 * All four DEVICE pointers. */
int icon_velocity_tendencies(icon_dycore_t* dycore, const double* vn, const double* w,
                             double* ddt_vn, double* ddt_w);

/* The reference state the dycore derived (HOST outputs, [nlev] each):
 * theta_ref and exner_ref at full levels; exner_ref is in exact discrete
 * hydrostatic balance with theta_ref on this vertical grid.  Over terrain the
 * reference state differs by column: ICON_ERR_UNSUPPORTED (use
 * icon_dycore_reference_columns). */
int icon_dycore_reference_state(const icon_dycore_t* dycore, double* theta_ref,
                                double* exner_ref);
/* The reference state per column (HOST outputs [n_cells*nlev] each, level-
 * contiguous): each column's own over terrain, the same profile in every
 * column over flat ground. */
int icon_dycore_reference_columns(const icon_dycore_t* dycore, double* theta_ref, double* exner_ref);

/* Diagnostics of a DEVICE state (outside the step):
 *   ps   [n_cells] DEVICE or NULL: surface pressure, Pa (exner at the ground
 *        extrapolated hydrostatically from the lowest level with its theta_v);
 *   t850 [n_cells] DEVICE or NULL: temperature at 850 hPa, K (linear in ln p);
 *   mass HOST scalar or NULL: total mass sum_c A_c sum_k rho dz, kg, summed in
 *        a fixed order (bitwise reproducible).
 * Returns ICON_ERR_NUMERIC when vn, w, rho, exner or theta_v holds a NaN or
 * an infinity (the outputs are still written); ICON_ERR_ARG for a host state. */
int icon_dycore_diagnostics(icon_dycore_t* dycore, const icon_state_t* state, double* ps, double* t850,
                            double* mass);

/* Cell areas in m^2 (HOST output [n_cells]), for area-weighted statistics. */
int icon_grid_cell_areas(const icon_grid_t* grid, double* area);

/* Measurement aid: run nsteps full steps on a DEVICE state (kernel by
 * kernel, not as a graph) with a CUDA event pair around every kernel launch
 * on the dycore's stream, then synchronize and report per kernel name:
 *   names    [max_kernels*64] NUL-terminated names (host buffer)
 *   launches [max_kernels]    number of launches
 *   ms       [max_kernels]    summed device time in milliseconds
 *   *n_kernels                number of distinct kernels reported
 * The state advances by nsteps steps.  Errors: ICON_ERR_ARG (NULL, host
 * state, max_kernels too small), ICON_ERR_CUDA. */
int icon_dycore_profile(icon_dycore_t* dycore, const icon_state_t* state, int32_t nsteps,
                        int32_t max_kernels, char* names, int32_t* launches, double* ms,
                        int32_t* n_kernels);

/* Verification aid (stage-level comparison, Sec. 4.4): copy the internal
 * work field `name` as it stands after the last call (values of the last
 * corrector where a field is reused) to dst (DEVICE pointer, `bytes` long,
 * layout as the state, element type double in FP64 mode and float for the
 * stencil fields and the predicted w in mixed mode, where div_m, div_t, rho_p
 * and theta_p hold double-word pairs (float hi, float lo; value hi + lo) in
 * 8-byte slots).  Names: vt, ekin_e (twice the kinetic energy, vn^2 + vt^2), ddt_vn0, ddt_vn1,
 * rho_e, theta_e, hpg, vn_p, divd, divd2, ddt_w0, ddt_w1, grad4, div_m,
 * div_t, w_p, rho_p, theta_p.  Errors: ICON_ERR_ARG (unknown name, bytes too
 * small), ICON_ERR_CUDA. */
int icon_dycore_debug_field(icon_dycore_t* dycore, const char* name, void* dst, int64_t bytes);

/* The launch shapes in use (picked by the autotuner when params.autotune is
 * set): writes a NUL-terminated text "name=threads,...;column_chunk=K" of at
 * most len bytes into buf (HOST).  The autotuner runs one step of every
 * kernel on a temporary uniform state at create time with each candidate
 * (128, 256, 512 threads per CTA for the stencils; 4, 6 or 8 levels per
 * shared-memory chunk for the column solve) and keeps the fastest per kernel. */
int icon_dycore_launch_config(const icon_dycore_t* dycore, char* buf, int32_t len);

/* Block until all work enqueued by this dycore has finished. */
int icon_dycore_synchronize(icon_dycore_t* dycore);

/* Checkpoint and restart of a state (DEVICE or HOST pointers, as for
 * icon_dycore_step; not mixed).  icon_dycore_save waits for the dycore's
 * enqueued work, then writes the file `path`: a 64-byte header (magic
 * "ICONDYCK", format version 1, nlev, n_cells, n_edges, payload size, FNV-1a
 * checksum of the payload's 64-bit words) followed by vn, w, rho, exner,
 * theta_v and exner_pr as FP64 in the state's layout, host byte order
 * (little-endian).  icon_dycore_load reads such a file into the state; it
 * checks the magic, the version, the sizes against this dycore's and the
 * checksum over the whole payload before it writes any field, so a refused
 * file leaves the state as it was.  A step from a loaded state equals the
 * step from the saved one bit for bit.  Errors: ICON_ERR_ARG (NULL argument,
 * NULL field, mixed pointers, a file that cannot be opened, written or read,
 * of another grid or damaged), ICON_ERR_CUDA. */
int icon_dycore_save(icon_dycore_t* dycore, const icon_state_t* state, const char* path);
int icon_dycore_load(icon_dycore_t* dycore, const icon_state_t* state, const char* path);

/* Sizes: nlev, n_cells, n_edges, n_verts (any output pointer may be NULL). */
int icon_dycore_sizes(const icon_dycore_t* dycore, int32_t* nlev, int32_t* n_cells,
                      int32_t* n_edges, int32_t* n_verts);

/*
 * Allocation-free vertically implicit column solve.  The paper has no
 * counterpart: this entry point is for callers that cannot allocate device
 * memory when they call -- typically a host model that reserved nearly all
 * device memory for its own arrays at start-up, so that the work arrays of a
 * whole step, which icon_dycore_create allocates, no longer fit.  Such a
 * caller can still run this solve on arrays it owns.
 *
 * It runs the same column kernel as icon_nh_solve (one thread per column,
 * Thomas elimination, Rayleigh damping, back-substitution, linearised
 * equation of state) for n_cols independent columns of nlev levels:
 *   z_ifc [nlev+1] HOST, half-level heights as for icon_dycore_create; read
 *          during the call only (it is passed to the GPU by value);
 *   p      the scheme parameters (dtime/ndyn_substeps is the time step of the
 *          solve; stream and synchronous are honoured; precision FP64 solves
 *          in FP64, MIXED in the mixed mode's double-word FP32 arithmetic,
 *          about 48 significant bits, on FP64 inputs and outputs; any other
 *          precision is refused);
 * DEVICE inputs, level-contiguous like the state:
 *   w [n_cols*(nlev+1)], rho, exner, theta_v [n_cols*nlev]  state at the
 *          start of the substep;
 *   ddt_w0 [n_cols*(nlev+1)]  explicit w tendency;
 *   div_m, div_t [n_cols*nlev]  horizontal divergences of the mass and
 *          rho*theta_v fluxes;
 *   rho_pred, theta_pred [n_cols*nlev], ddt_w1 [n_cols*(nlev+1)]  the
 *          predicted state and its w tendency for the corrector form
 *          (half levels from 0.6 now + 0.4 predicted, tendency 0.25 ddt_w0 +
 *          0.75 ddt_w1); all three NULL for the predictor form.
 * DEVICE outputs (may alias the corresponding inputs): w_new, rho_new,
 *   exner_new, theta_new.
 * Scratch: one file-scope static device array of 64 MiB, held by every GPU
 * that loads this library until the process exits; it limits a call to
 * nlev <= 256 and n_cols*(nlev+1) <= 1 047 232 column-levels (at nlev = 90:
 * 11 508 columns); larger calls return ICON_ERR_ARG before any GPU work.
 * No cudaMalloc, cudaFree or other allocating call is made.  The vertical
 * metrics are computed on the device, by a one-thread kernel on the same
 * stream, from z_ifc and the scalars passed by value.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress)
 * and sets the kernel's shared-memory limit.  All calls share the array and
 * it keeps the last call's contents (every value a call reads is written
 * earlier in the same call, so nothing needs clearing); calls whose GPU work
 * overlaps -- on different streams, or from different threads -- race on it
 * and must be serialised by the caller.
 * Errors: ICON_ERR_ARG (NULL, sizes beyond the limit, bad z_ifc, time step
 * or precision), ICON_ERR_CUDA.
 */
int icon_column_solve_noalloc(int32_t n_cols, int32_t nlev, const double* z_ifc,
                              const icon_dycore_params_t* p, const double* w, const double* rho,
                              const double* exner, const double* theta_v, const double* rho_pred,
                              const double* theta_pred, const double* ddt_w0, const double* ddt_w1,
                              const double* div_m, const double* div_t, double* w_new,
                              double* rho_new, double* exner_new, double* theta_new);

/*
 * Learned corrector network (an extension beyond the paper's step, which has
 * no learned component): a 3-layer MLP
 *   y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3,  GELU(u) = u Phi(u) (erf form),
 * BF16 weights and activations with FP32 accumulation on the tensor cores,
 * FP32 master weights, trained on the GPU with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on the mean squared error.  Parameters are exchanged as one FP32
 * host array: W1 [n_hidden][n_in], b1 [n_hidden], W2 [n_hidden][n_hidden],
 * b2, W3 [n_out][n_hidden], b3 (each W row-major, output index first).
 * Inputs x [batch][n_in] and outputs/targets [batch][n_out] are FP32 DEVICE
 * arrays; batch <= max_batch, and a multiple of 64 for backward/training.
 */
typedef struct icon_mlp icon_mlp_t;  /* opaque */
int icon_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, icon_mlp_t** out);
int icon_mlp_destroy(icon_mlp_t* mlp);          /* NULL-safe */
int64_t icon_mlp_param_count(const icon_mlp_t* mlp);
/* Set all parameters (resets the Adam moments); get parameters / the last gradients. */
int icon_mlp_set_params(icon_mlp_t* mlp, const float* params, int64_t n);
int icon_mlp_get_params(const icon_mlp_t* mlp, float* params, int64_t n);
int icon_mlp_get_grads(const icon_mlp_t* mlp, float* grads, int64_t n);
/* Forward pass (keeps the activations of the batch for a following backward). */
int icon_mlp_forward(icon_mlp_t* mlp, const float* x, int32_t batch, float* y, void* stream);
/* Gradients of all parameters for dL/dy [batch][n_out] (DEVICE), after a forward
 * on the same batch; read them with icon_mlp_get_grads. */
int icon_mlp_backward(icon_mlp_t* mlp, const float* dy, int32_t batch, void* stream);
/* One Adam update with the last gradients. */
int icon_mlp_adam(icon_mlp_t* mlp, float lr, float beta1, float beta2, float eps, void* stream);
/* forward + MSE loss against target + backward + Adam; *loss (HOST, may be NULL)
 * receives the batch's mean squared error before the update. */
int icon_mlp_train_step(icon_mlp_t* mlp, const float* x, const float* target, int32_t batch, float lr,
                        double* loss, void* stream);

/* Normalisation statistics used by icon_dycore_step_learned (HOST FP32 arrays,
 * copied): the network's input is (x - x_mean) / x_std per feature, and an
 * output y stands for the physical increment y y_std + y_mean. */
int icon_mlp_set_normalization(icon_mlp_t* mlp, const float* x_mean, const float* x_std, const float* y_mean,
                               const float* y_std);
/* The statistics in use (HOST outputs [n_in], [n_in], [n_out], [n_out]);
 * ICON_ERR_ARG when the network has none. */
int icon_mlp_get_normalization(const icon_mlp_t* mlp, float* x_mean, float* x_std, float* y_mean, float* y_std);
/* Training statistics on the GPU: the mean and the sample standard deviation
 * (divisor rows - 1, FP64 accumulation in a fixed order) of every feature of
 * the training rows x [rows][n_in] and targets y [rows][n_out] (DEVICE, FP32),
 * a standard deviation below rel_floor times the largest of its group raised
 * to that floor (groups: HOST int32 arrays of the groups' first features,
 * ascending from 0; a group runs to the next one's start, the last to the
 * end), set as the network's normalisation, and the normalised rows written
 * to xn [rows][n_in] and yn [rows][n_out] (DEVICE).  Allocates and frees its
 * own scratch; synchronises the stream before returning.
 * Errors: ICON_ERR_ARG (NULL, rows < 2, bad groups), ICON_ERR_CUDA. */
int icon_mlp_fit_normalization(icon_mlp_t* mlp, const float* x, const float* y, int64_t rows, const int32_t* x_groups,
                               int32_t n_x_groups, const int32_t* y_groups, int32_t n_y_groups, float rel_floor,
                               float* xn, float* yn, void* stream);
/* One training step (as icon_mlp_train_step) on a random batch of `batch`
 * rows of the normalised training set xn [rows][n_in], yn [rows][n_out]
 * (DEVICE): batch row i is training row splitmix64(seed + 2^32 step + i) mod
 * rows (SplitMix64: a counter-based generator, so the batches need no host
 * work and step s draws the same rows whatever ran before).  batch a multiple
 * of 64 up to max_batch. */
int icon_mlp_train_step_sampled(icon_mlp_t* mlp, const float* xn, const float* yn, int64_t rows, int32_t batch,
                                uint64_t seed, int64_t step, float lr, double* loss, void* stream);

/*
 * Learned corrector on the state after a step with fewer acoustic substeps
 * (Sec. 3.2's substep loop with ndyn_substeps reduced).  Column features of a
 * cell, [nc][5 nlev] (FP32, DEVICE): w at full levels (mean of the two half
 * levels), exner - exner_ref, theta_v - theta_ref, and the cell velocity's east
 * and north components (Perot reconstruction from vn).  Edge features
 * [ne][11 nlev]: the column features of e2c[0] and of e2c[1], then vn.
 * Column outputs [nc][3 nlev - 1]: increments of w at the interior half levels
 * 1..nlev-1, of exner and of theta_v; edge outputs [ne][nlev]: increments of vn.
 * rho and exner_pr are never changed, so the mass budget of the reduced step is
 * kept exactly.
 */
/* Raw (unnormalised) features of a DEVICE state into DEVICE arrays. */
int icon_corrector_features(icon_dycore_t* d, const icon_state_t* s, float* col_x, float* edge_x);
/* Raw training targets plain - reduced into DEVICE arrays col_y [nc][3 nlev - 1]
 * and edge_y [ne][nlev]; both states on the device. */
int icon_corrector_targets(icon_dycore_t* d, const icon_state_t* reduced, const icon_state_t* plain, float* col_y,
                           float* edge_y);
/*
 * One learned step of a DEVICE state, in place: keep the input, run the step of
 * `reduced` (fewer substeps), apply col_net (5 nlev -> 3 nlev - 1) and edge_net
 * (11 nlev -> nlev) over all cells and edges in chunks of their max_batch,
 * then check.  The check is the larger of the two networks' RMS normalised
 * increments; if it is not finite (a non-finite increment, corrected value or
 * rho is found) or above max_norm, the input is restored and the step of
 * `plain` taken instead (*used_fallback = 1).  *norm (may be NULL) receives the
 * check value.  Both dycores share the grid and nlev; both networks must carry
 * normalisation statistics.  Synchronises the stream once (the check's 16-byte
 * read).  Errors: ICON_ERR_ARG for NULL, host state, mismatched dycores or
 * network shapes; ICON_ERR_CUDA.
 */
int icon_dycore_step_learned(icon_dycore_t* reduced, icon_dycore_t* plain, icon_mlp_t* col_net,
                             icon_mlp_t* edge_net, const icon_state_t* s, double max_norm, int32_t* used_fallback,
                             double* norm);

/*
 * Per-kernel profile of any sequence of calls on this thread (Sec. 4.3's
 * execution profile of a substep, Sec. 5.1's synchronised timers): between
 * icon_profile_begin and icon_profile_end every kernel launch of the library is
 * bracketed by a CUDA event pair on its stream (steps run without their graph
 * meanwhile, so each kernel is seen).  icon_profile_end synchronises the device
 * and fills, for up to max_kernels distinct kernels, names[64 j] (NUL-
 * terminated), launches[j] and summed milliseconds ms[j]; *n_kernels = count.
 * Errors: ICON_ERR_ARG when no profile (or already one) is open on this thread,
 * for NULL outputs or too small max_kernels.
 */
int icon_profile_begin(void);
int icon_profile_end(int32_t max_kernels, char* names, int32_t* launches, double* ms, int32_t* n_kernels);

/*
 * ICON's nproma-blocked arrays (Sec. 4.3: the host model hands the dycore its
 * own arrays).  A blocked field of n points and nlev_x levels is the Fortran
 * array X(nproma, nlev_x, nblks), nblks = ceil(n / nproma): point h = jb*nproma
 * + jc (0-based) at level k sits at offset jc + nproma*(k + nlev_x*jb); the
 * pad points of the last block are neither read nor written.  The library's
 * own layout is level-contiguous, X[h*nlev_x + k].  These calls convert all six
 * state fields on the device (a shared-memory tiled transpose, about the cost
 * of copying the state once each way: not zero-copy).  All arrays DEVICE;
 * source and destination must not share an array; nproma >= 1 with at most
 * 65535 blocks.  Errors: ICON_ERR_ARG, ICON_ERR_CUDA.
 */
int icon_state_from_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* blocked, const icon_state_t* state);
int icon_state_to_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* state, const icon_state_t* blocked);
/* One step (as icon_dycore_step) of a blocked state, in place: converted into
 * the dycore's own device copy, stepped, converted back. */
int icon_dycore_step_blocked(icon_dycore_t* d, int32_t nproma, const icon_state_t* blocked);

/* Message of the last failing call on this thread ("" if none). */
const char* icon_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ICON_DYCORE_H */
