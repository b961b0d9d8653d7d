"""FP64 CPU oracle of the learned corrector's data path (test infrastructure only).

Row A13.  The corrector is an extension beyond the paper (its step has no
learned part):
after a step with fewer acoustic substeps (Sec. 3.2's substep loop with a
smaller ndyn_substeps) two networks propose increments towards the plain step
taken from the same input.  Definitions, in the order the step applies them:

* column features of cell c, five blocks of nlev values (levels top first):
  w at full levels (w_k + w_{k+1}) / 2, exner - exner_ref, theta_v - theta_ref
  (the reference state of the cell's own column over terrain),
  and the east and north components of the Perot cell velocity
  (1/A_c) sum_e s l_e vn_e (x_e - x_c) with east = unit(z x r_c), north = r_c x east;
* edge features of edge e: the column features of e2c[e,0], then those of
  e2c[e,1], then vn_e over the levels (11 nlev values);
* inputs are normalised per feature, x_n = (x - x_mean) / x_std; an output y
  stands for the increment y y_std + y_mean;
* column outputs (3 nlev - 1): increments of w at the interior half levels
  1..nlev-1, of exner and of theta_v; edge outputs (nlev): increments of vn;
  rho and exner_pr are never changed;
* the check value is the larger of the two networks' RMS normalised outputs;
  a value that is not finite (or a corrected field or rho that is not finite)
  or above max_norm rejects the correction, and the plain step from the saved
  input is taken instead.
"""
import numpy as np

from . import mlp


def east_north(C):
    """Unit east and north vectors at the unit position vectors C [n, 3]."""
    east = np.cross(np.array([0.0, 0.0, 1.0]), C)
    east /= np.linalg.norm(east, axis=1)[:, None]
    north = np.cross(C, east)
    return east, north


def column_features(dycore, st):
    """[nc, 5 nlev] float64 features of the state (see the module docstring)."""
    g = dycore.g
    th_ref, ex_ref = dycore.reference_state()
    w = st["w"]
    u3 = dycore.perot_cell(st["vn"])
    east, north = east_north(g.C)
    u = np.einsum("ckx,cx->ck", u3, east)
    v = np.einsum("ckx,cx->ck", u3, north)
    if ex_ref.ndim == 1:      # one profile for all columns (flat ground); per column over terrain
        th_ref, ex_ref = th_ref[None, :], ex_ref[None, :]
    return np.concatenate([0.5 * (w[:, :-1] + w[:, 1:]), st["exner"] - ex_ref,
                           st["theta_v"] - th_ref, u, v], axis=1)


def edge_features(dycore, st, col_x=None):
    """[ne, 11 nlev] float64 features: the two adjacent columns, then vn."""
    g = dycore.g
    if col_x is None:
        col_x = column_features(dycore, st)
    return np.concatenate([col_x[g.e2c[:, 0]], col_x[g.e2c[:, 1]], st["vn"]], axis=1)


def targets(reduced, plain):
    """Training targets plain - reduced: column [nc, 3 nlev - 1], edge [ne, nlev]."""
    dw = plain["w"][:, 1:-1] - reduced["w"][:, 1:-1]
    col = np.concatenate([dw, plain["exner"] - reduced["exner"], plain["theta_v"] - reduced["theta_v"]], axis=1)
    return col, plain["vn"] - reduced["vn"]


def network(params, dims, stats, x):
    """Denormalised increments of a network on raw features x.
    dims = (n_in, n_hidden, n_out); stats = (x_mean, x_std, y_mean, y_std).
    Returns (increments, normalised outputs)."""
    xm, xs, ym, ys = [np.asarray(a, dtype=np.float64) for a in stats]
    y, _ = mlp.forward(params, (x - xm) / xs, *dims)
    return y * ys + ym, y


def apply(st, col_inc, edge_inc):
    """The corrected state: increments added to interior w, exner, theta_v and vn."""
    out = {k: v.copy() for k, v in st.items()}
    nlev = st["exner"].shape[1]
    out["w"][:, 1:-1] += col_inc[:, :nlev - 1]
    out["exner"] += col_inc[:, nlev - 1:2 * nlev - 1]
    out["theta_v"] += col_inc[:, 2 * nlev - 1:]
    out["vn"] += edge_inc
    return out


def check_value(col_y, edge_y, corrected):
    """max of the two RMS normalised outputs; NaN when anything corrected (or rho) is not finite."""
    r = max(np.sqrt(np.mean(col_y ** 2)), np.sqrt(np.mean(edge_y ** 2)))
    fields = ("vn", "w", "exner", "theta_v", "rho")
    if not all(np.all(np.isfinite(corrected[k])) for k in fields):
        return float("nan")
    return float(r)


def step_learned(reduced, plain, col_net, edge_net, st, max_norm):
    """One learned step.  reduced/plain are oracle Dycore objects sharing the grid;
    col_net and edge_net are (params, dims, stats).  Returns (state, used_fallback, check value)."""
    sr = reduced.step(st)
    cx = column_features(reduced, sr)
    ex = edge_features(reduced, sr, cx)
    col_inc, col_y = network(*col_net, cx)
    edge_inc, edge_y = network(*edge_net, ex)
    corrected = apply(sr, col_inc, edge_inc)
    r = check_value(col_y, edge_y, corrected)
    if not (r <= max_norm):
        return plain.step(st), True, r
    return corrected, False, r
