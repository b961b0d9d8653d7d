"""Python binding of libicondycore (GB300 ICON-type nonhydrostatic dycore).

Argument marshalling only: every computation of the dycore runs in the CUDA
kernels behind the C-ABI declared in ``include/icon_dycore.h``.  The entry
points keep the C names (``icon_grid_create``, ``icon_dycore_create``,
``icon_dycore_step``, ``icon_nh_solve``, ``icon_nh_diff``, ...); ``Grid`` and
``Dycore`` below only own the handles and pass tensor pointers.

Fields are passed as torch tensors (device pointers, no copies) or as
C-contiguous numpy float64 arrays (host pointers; the library copies them in
and out around the call).  Importing this module fails if the shared library
has not been built (``python -m paper_2608_21150_gb300.build``): there is no
fallback implementation.
"""
import ctypes
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(
        "libicondycore.so is not built; run `python -m paper_2608_21150_gb300.build` "
        "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIB)

ICON_OK = 0
ICON_ERR_ARG = -1
ICON_ERR_CUDA = -2
ICON_ERR_GRID = -3
ICON_ERR_NUMERIC = -4
ICON_ERR_UNSUPPORTED = -5
ICON_PREC_FP64 = 0
ICON_PREC_MIXED = 1
ICON_PREC_MIXED_F64COL = 2

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class icon_grid_desc_t(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("n_verts", ctypes.c_int32),
                ("index_base", ctypes.c_int32), ("sphere_radius", ctypes.c_double),
                ("c2v", _i32p), ("c2e", _i32p), ("e2c", _i32p), ("e2v", _i32p), ("v2e", _i32p),
                ("v2c", _i32p), ("cell_xyz", _f64p), ("vert_xyz", _f64p), ("edge_xyz", _f64p)]


class icon_dycore_params_t(ctypes.Structure):
    _fields_ = [("dtime", ctypes.c_double), ("ndyn_substeps", ctypes.c_int32),
                ("grav", ctypes.c_double), ("rd", ctypes.c_double), ("cpd", ctypes.c_double),
                ("p00", ctypes.c_double), ("omega", ctypes.c_double),
                ("vwind_impl_wgt", ctypes.c_double), ("wgt_nnow_vel", ctypes.c_double),
                ("wgt_nnew_vel", ctypes.c_double), ("wgt_nnow_rth", ctypes.c_double),
                ("wgt_nnew_rth", ctypes.c_double), ("exner_exfac", ctypes.c_double),
                ("divdamp_fac", ctypes.c_double), ("divflux_fac", ctypes.c_double),
                ("rayleigh_coeff", ctypes.c_double),
                ("damp_height", ctypes.c_double), ("hdiff_smag_fac", ctypes.c_double),
                ("hdiff_k4", ctypes.c_double), ("hdiff_w_k4", ctypes.c_double),
                ("hdiff_temp", ctypes.c_int32), ("ref_T0", ctypes.c_double),
                ("precision", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("synchronous", ctypes.c_int32), ("stream", ctypes.c_void_p), ("column_chunk", ctypes.c_int32),
                ("steep_hpg", ctypes.c_int32), ("hdiff_tenh_fac", ctypes.c_double),
                ("hdiff_tenh_thresh", ctypes.c_double), ("hdiff_tenh_levels", ctypes.c_int32),
                ("fused_advection", ctypes.c_int32)]


class icon_state_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("vn", "w", "rho", "exner", "theta_v", "exner_pr")]


STATE_FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")

_sig = {
    "icon_grid_create": (ctypes.c_int, [ctypes.POINTER(icon_grid_desc_t), ctypes.POINTER(ctypes.c_void_p)]),
    "icon_grid_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "icon_dycore_params_default": (None, [ctypes.POINTER(icon_dycore_params_t)]),
    "icon_dycore_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _f64p,
                                          ctypes.POINTER(icon_dycore_params_t),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "icon_dycore_create_terrain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _f64p,
                                                  ctypes.POINTER(icon_dycore_params_t),
                                                  ctypes.POINTER(ctypes.c_void_p)]),
    "icon_dycore_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "icon_dycore_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t)]),
    "icon_nh_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t)]),
    "icon_nh_diff": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t)]),
    "icon_velocity_tendencies": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4),
    "icon_dycore_reference_state": (ctypes.c_int, [ctypes.c_void_p, _f64p, _f64p]),
    "icon_dycore_reference_columns": (ctypes.c_int, [ctypes.c_void_p, _f64p, _f64p]),
    "icon_dycore_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "icon_dycore_launch_config": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32]),
    "icon_dycore_debug_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_int64]),
    "icon_dycore_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t), ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_char_p, _i32p, _f64p, _i32p]),
    "icon_dycore_sizes": (ctypes.c_int, [ctypes.c_void_p] + [_i32p] * 4),
    "icon_dycore_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p]),
    "icon_dycore_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p]),
    "icon_last_error": (ctypes.c_char_p, []),
    "icon_dycore_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t), ctypes.c_void_p,
                                               ctypes.c_void_p, _f64p]),
    "icon_grid_cell_areas": (ctypes.c_int, [ctypes.c_void_p, _f64p]),
    "icon_mlp_create": (ctypes.c_int, [ctypes.c_int32] * 4 + [ctypes.POINTER(ctypes.c_void_p)]),
    "icon_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "icon_mlp_param_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "icon_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "icon_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "icon_mlp_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "icon_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "icon_mlp_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "icon_mlp_adam": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_float] * 4 + [ctypes.c_void_p]),
    "icon_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_float, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "icon_mlp_set_normalization": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_float)] * 4),
    "icon_mlp_get_normalization": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_float)] * 4),
    "icon_mlp_fit_normalization": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                  _i32p, ctypes.c_int32, _i32p, ctypes.c_int32, ctypes.c_float,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "icon_mlp_train_step_sampled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                   ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_float,
                                                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "icon_corrector_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t), ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "icon_corrector_targets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(icon_state_t),
                                              ctypes.POINTER(icon_state_t), ctypes.c_void_p, ctypes.c_void_p]),
    "icon_dycore_step_learned": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.POINTER(icon_state_t), ctypes.c_double,
                                                _i32p, _f64p]),
    "icon_state_from_blocked": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(icon_state_t),
                                               ctypes.POINTER(icon_state_t)]),
    "icon_state_to_blocked": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(icon_state_t),
                                             ctypes.POINTER(icon_state_t)]),
    "icon_dycore_step_blocked": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(icon_state_t)]),
    "icon_profile_begin": (ctypes.c_int, []),
    "icon_profile_end": (ctypes.c_int, [ctypes.c_int32, ctypes.c_char_p, _i32p, _f64p, _i32p]),
    "icon_column_solve_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _f64p,
                                                 ctypes.POINTER(icon_dycore_params_t)] + [ctypes.c_void_p] * 14),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class IconError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


def _check(rc):
    if rc != ICON_OK:
        raise IconError(rc, icon_last_error().decode())
    return rc


def default_params(**overrides):
    p = icon_dycore_params_t()
    icon_dycore_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(x):
    """Raw pointer of a torch tensor or a numpy array (must be contiguous float64)."""
    if isinstance(x, np.ndarray):
        if not (x.flags["C_CONTIGUOUS"] and x.dtype == np.float64):
            raise ValueError("numpy fields must be C-contiguous float64")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor fields must be contiguous")
    return x.data_ptr()


def column_solve_noalloc(z_ifc, params, w, rho, exner, theta_v, ddt_w0, div_m, div_t, w_new, rho_new,
                         exner_new, theta_new, rho_pred=None, theta_pred=None, ddt_w1=None):
    """icon_column_solve_noalloc on device tensors; the three optional fields
    select the corrector form.  ``params`` is an icon_dycore_params_t or a
    dict of overrides."""
    if params is None or isinstance(params, dict):
        params = default_params(**(params or {}))
    z = np.ascontiguousarray(z_ifc, dtype=np.float64)
    n_cols = rho.shape[0] if rho.dim() == 2 else rho.numel() // (z.size - 1)
    opt = [None if x is None else _ptr(x) for x in (rho_pred, theta_pred, ddt_w1)]
    _check(icon_column_solve_noalloc(n_cols, z.size - 1, z.ctypes.data_as(_f64p), ctypes.byref(params),
                                     _ptr(w), _ptr(rho), _ptr(exner), _ptr(theta_v), opt[0], opt[1],
                                     _ptr(ddt_w0), opt[2], _ptr(div_m), _ptr(div_t), _ptr(w_new),
                                     _ptr(rho_new), _ptr(exner_new), _ptr(theta_new)))


class MLP:
    """Owns an icon_mlp_t (the learned corrector's network); tensors are float32 on the device."""

    def __init__(self, n_in, n_hidden, n_out, max_batch):
        h = ctypes.c_void_p()
        _check(icon_mlp_create(n_in, n_hidden, n_out, max_batch, ctypes.byref(h)))
        self.handle = h
        self.n_in, self.n_hidden, self.n_out, self.max_batch = n_in, n_hidden, n_out, max_batch
        self.n_params = icon_mlp_param_count(h)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(icon_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    def _get(self, fn):
        p = np.empty(self.n_params, dtype=np.float32)
        _check(fn(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def params(self):
        return self._get(icon_mlp_get_params)

    def grads(self):
        return self._get(icon_mlp_get_grads)

    def forward(self, x, y, stream=None):
        _check(icon_mlp_forward(self.handle, _ptr(x), x.shape[0], _ptr(y), stream))

    def backward(self, dy, stream=None):
        _check(icon_mlp_backward(self.handle, _ptr(dy), dy.shape[0], stream))

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(icon_mlp_adam(self.handle, lr, beta1, beta2, eps, stream))

    def set_normalization(self, x_mean, x_std, y_mean, y_std):
        """Input/output statistics (host arrays) used by the learned step."""
        fp = ctypes.POINTER(ctypes.c_float)
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (x_mean, x_std, y_mean, y_std)]
        if arrs[0].size != self.n_in or arrs[1].size != self.n_in or arrs[2].size != self.n_out \
                or arrs[3].size != self.n_out:
            raise ValueError("normalisation sizes must be n_in, n_in, n_out, n_out")
        _check(icon_mlp_set_normalization(self.handle, *[a.ctypes.data_as(fp) for a in arrs]))
        self.normalization = tuple(arrs)

    def train_step(self, x, target, lr, stream=None):
        loss = ctypes.c_double()
        _check(icon_mlp_train_step(self.handle, _ptr(x), _ptr(target), x.shape[0], lr, ctypes.byref(loss), stream))
        return loss.value

    def get_normalization(self):
        """The statistics in use (host float32 arrays x_mean, x_std, y_mean, y_std)."""
        fp = ctypes.POINTER(ctypes.c_float)
        arrs = [np.empty(n, dtype=np.float32) for n in (self.n_in, self.n_in, self.n_out, self.n_out)]
        _check(icon_mlp_get_normalization(self.handle, *[a.ctypes.data_as(fp) for a in arrs]))
        return tuple(arrs)

    def fit_normalization(self, x, y, x_groups, y_groups, rel_floor, xn, yn, stream=None):
        """icon_mlp_fit_normalization on device tensors x, y (and outputs xn, yn)."""
        xg = np.ascontiguousarray(x_groups, dtype=np.int32)
        yg = np.ascontiguousarray(y_groups, dtype=np.int32)
        _check(icon_mlp_fit_normalization(self.handle, _ptr(x), _ptr(y), x.shape[0], xg.ctypes.data_as(_i32p),
                                          xg.size, yg.ctypes.data_as(_i32p), yg.size, rel_floor, _ptr(xn), _ptr(yn),
                                          stream))
        self.normalization = self.get_normalization()

    def train_step_sampled(self, xn, yn, batch, seed, step, lr, stream=None):
        """icon_mlp_train_step_sampled: one step on a random batch of the normalised rows."""
        loss = ctypes.c_double()
        _check(icon_mlp_train_step_sampled(self.handle, _ptr(xn), _ptr(yn), xn.shape[0], batch, seed, step, lr,
                                           ctypes.byref(loss), stream))
        return loss.value

    def close(self):
        if self.handle:
            icon_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Profile:
    """Context manager around icon_profile_begin/end: per-kernel launches and
    milliseconds of every library kernel launched on this thread inside the
    block, as ``{name: (launches, ms)}`` in ``.kernels`` on exit."""

    def __enter__(self):
        _check(icon_profile_begin())
        self.kernels = {}
        return self

    def __exit__(self, *exc):
        cap = 128
        names = ctypes.create_string_buffer(64 * cap)
        launches = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int32()
        _check(icon_profile_end(cap, names, launches, ms, ctypes.byref(n)))
        self.kernels = {names.raw[64 * j:64 * j + 64].split(b"\0")[0].decode(): (launches[j], ms[j])
                        for j in range(n.value)}
        return False


def step_learned(reduced, plain, col_net, edge_net, st, max_norm):
    """icon_dycore_step_learned: one step of `reduced` plus the learned increments,
    or the step of `plain` when the check fails.  Returns (used_fallback, norm)."""
    s = Dycore._state(st)
    fb = ctypes.c_int32()
    nrm = ctypes.c_double()
    _check(icon_dycore_step_learned(reduced.handle, plain.handle, col_net.handle, edge_net.handle, ctypes.byref(s),
                                    max_norm, ctypes.byref(fb), ctypes.byref(nrm)))
    return bool(fb.value), nrm.value


class Grid:
    """Owns an icon_grid_t built from raw connectivity and coordinates."""

    def __init__(self, grid, radius=6.371229e6, index_base=0):
        keep = {}

        def i32(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            keep[id(a)] = a
            return a.ctypes.data_as(_i32p)

        def f64(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep[id(a)] = a
            return a.ctypes.data_as(_f64p)

        off = index_base
        d = icon_grid_desc_t(grid.n_cells, grid.n_edges, grid.n_verts, index_base, radius,
                             i32(grid.c2v + off), i32(grid.c2e + off), i32(grid.e2c + off),
                             i32(grid.e2v + off), i32(grid.v2e + off), i32(grid.v2c + off),
                             f64(grid.cell_xyz), f64(grid.vert_xyz), f64(grid.edge_xyz))
        h = ctypes.c_void_p()
        _check(icon_grid_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_cells, self.n_edges, self.n_verts = grid.n_cells, grid.n_edges, grid.n_verts

    def cell_areas(self):
        a = np.empty(self.n_cells)
        _check(icon_grid_cell_areas(self.handle, a.ctypes.data_as(_f64p)))
        return a

    def close(self):
        if self.handle:
            icon_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dycore:
    """Owns an icon_dycore_t.  ``params`` is an icon_dycore_params_t or a dict of overrides."""

    def __init__(self, grid: Grid, z_ifc, params=None, stream=None):
        if params is None or isinstance(params, dict):
            params = default_params(**(params or {}))
        if stream is not None:
            params.stream = stream
        z = np.ascontiguousarray(z_ifc, dtype=np.float64)
        h = ctypes.c_void_p()
        # one column of heights: flat ground; [n_cells, nlev+1]: terrain-following
        self.terrain = z.ndim == 2
        if self.terrain:
            if z.shape[0] != grid.n_cells:
                raise ValueError("terrain heights must be [n_cells, nlev+1]")
            self.nlev = z.shape[1] - 1
            _check(icon_dycore_create_terrain(grid.handle, self.nlev, z.ctypes.data_as(_f64p), ctypes.byref(params),
                                              ctypes.byref(h)))
        else:
            self.nlev = z.size - 1
            _check(icon_dycore_create(grid.handle, self.nlev, z.ctypes.data_as(_f64p), ctypes.byref(params),
                                      ctypes.byref(h)))
        self.handle = h
        self.grid = grid
        self.params = params

    @staticmethod
    def _state(st):
        return icon_state_t(*[_ptr(st[n]) for n in STATE_FIELDS])

    def step(self, st):
        s = self._state(st)
        _check(icon_dycore_step(self.handle, ctypes.byref(s)))

    def nh_solve(self, st):
        s = self._state(st)
        _check(icon_nh_solve(self.handle, ctypes.byref(s)))

    def nh_diff(self, st):
        s = self._state(st)
        _check(icon_nh_diff(self.handle, ctypes.byref(s)))

    def velocity_tendencies(self, vn, w, ddt_vn, ddt_w):
        _check(icon_velocity_tendencies(self.handle, _ptr(vn), _ptr(w), _ptr(ddt_vn), _ptr(ddt_w)))

    def from_blocked(self, nproma, blocked, st):
        """ICON nproma-blocked device state -> the library's layout (device)."""
        a, b = self._state(blocked), self._state(st)
        _check(icon_state_from_blocked(self.handle, nproma, ctypes.byref(a), ctypes.byref(b)))

    def to_blocked(self, nproma, st, blocked):
        """The library's layout -> ICON nproma-blocked device state."""
        a, b = self._state(st), self._state(blocked)
        _check(icon_state_to_blocked(self.handle, nproma, ctypes.byref(a), ctypes.byref(b)))

    def step_blocked(self, nproma, blocked):
        """One step of an ICON nproma-blocked device state, in place."""
        a = self._state(blocked)
        _check(icon_dycore_step_blocked(self.handle, nproma, ctypes.byref(a)))

    def corrector_features(self, st, col_x, edge_x):
        """Raw corrector features of a device state: col_x [n_cells][5 nlev],
        edge_x [n_edges][11 nlev] (float32 device tensors)."""
        s = self._state(st)
        _check(icon_corrector_features(self.handle, ctypes.byref(s), _ptr(col_x), _ptr(edge_x)))

    def corrector_targets(self, reduced, plain, col_y, edge_y):
        """Raw corrector targets plain - reduced: col_y [n_cells][3 nlev - 1], edge_y [n_edges][nlev]."""
        a, b = self._state(reduced), self._state(plain)
        _check(icon_corrector_targets(self.handle, ctypes.byref(a), ctypes.byref(b), _ptr(col_y), _ptr(edge_y)))

    def reference_state(self):
        th = np.empty(self.nlev)
        ex = np.empty(self.nlev)
        _check(icon_dycore_reference_state(self.handle, th.ctypes.data_as(_f64p), ex.ctypes.data_as(_f64p)))
        return th, ex

    def reference_columns(self):
        """Reference theta_v and exner per column, [n_cells, nlev] each."""
        th = np.empty((self.grid.n_cells, self.nlev))
        ex = np.empty((self.grid.n_cells, self.nlev))
        _check(icon_dycore_reference_columns(self.handle, th.ctypes.data_as(_f64p), ex.ctypes.data_as(_f64p)))
        return th, ex

    def profile(self, st, nsteps):
        """Per-kernel launch counts and summed device milliseconds over nsteps steps
        (events around every launch); returns {name: (launches, ms)}."""
        s = self._state(st)
        cap = 64
        names = ctypes.create_string_buffer(64 * cap)
        launches = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int32()
        _check(icon_dycore_profile(self.handle, ctypes.byref(s), nsteps, cap, names, launches, ms,
                                   ctypes.byref(n)))
        return {names.raw[64 * j:64 * j + 64].split(b"\0")[0].decode(): (launches[j], ms[j])
                for j in range(n.value)}

    def diagnostics(self, st, ps=None, t850=None):
        """Fill the device tensors ps/t850 [n_cells] (if given) and return the total
        mass; raises IconError(ICON_ERR_NUMERIC) for a non-finite state."""
        s = self._state({k: st[k] for k in ("vn", "w", "rho", "exner", "theta_v")} | {"exner_pr": st["rho"]})
        m = ctypes.c_double()
        _check(icon_dycore_diagnostics(self.handle, ctypes.byref(s), None if ps is None else _ptr(ps),
                                       None if t850 is None else _ptr(t850), ctypes.byref(m)))
        return m.value

    def debug_field(self, name, out):
        """Copy the internal work field `name` into the device tensor `out`."""
        _check(icon_dycore_debug_field(self.handle, name.encode(), _ptr(out), out.numel() * out.element_size()))

    def save(self, st, path):
        """Write the state (device tensors or host arrays) to the checkpoint file `path`."""
        s = self._state(st)
        _check(icon_dycore_save(self.handle, ctypes.byref(s), os.fsencode(path)))

    def load(self, st, path):
        """Read the checkpoint file `path` into the state (device tensors or host arrays)."""
        s = self._state(st)
        _check(icon_dycore_load(self.handle, ctypes.byref(s), os.fsencode(path)))

    def launch_config(self):
        buf = ctypes.create_string_buffer(1024)
        _check(icon_dycore_launch_config(self.handle, buf, 1024))
        return buf.value.decode()

    def synchronize(self):
        _check(icon_dycore_synchronize(self.handle))

    def close(self):
        if self.handle:
            icon_dycore_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
