"""Probtest-style ensemble tolerances from the FP64 oracle (test
infrastructure only).

The paper's third verification level (Sec. 4.4) runs a reference ensemble of
the same experiment with randomly perturbed inputs, one random seed per
member, over 5-10 model steps (25-50 dycore substeps), and derives a
tolerance for every output field from it; a run passes when its differences
from the reference stay within those tolerances.  Reading used here (the
paper defers the details to the probtest tool):

* the reference is the unperturbed oracle run (the control);
* members start from the control's initial state with vn, rho, exner and
  theta_v perturbed by a relative amount eps (icon_inputs.perturb_state), the
  exner history re-derived from the perturbed exner;
* the difference of a state from the control is, per field, the maximum
  absolute difference over all points divided by the maximum magnitude of the
  control field (exner and theta_v as deviations from the reference profiles,
  the same norm as the parity tests);
* the spread of a field at step n is the largest such difference over the
  members; the tolerance is a fixed factor times the spread.
"""
import numpy as np

from icon_inputs import perturb_state

FIELDS = ("vn", "w", "rho", "exner", "theta_v")


def differences(a, b, dycore):
    """Per-field relative max-norm difference of state a from the control b.
    Sec. 4.4: probtest-style ensemble verification, a reading."""
    th_ref, ex_ref = dycore.reference_state()
    if ex_ref.ndim == 1:      # per column over terrain
        th_ref, ex_ref = th_ref[None, :], ex_ref[None, :]
    out = {}
    for k in FIELDS:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        if k == "exner":
            x, y = x - ex_ref, y - ex_ref
        if k == "theta_v":
            x, y = x - th_ref, y - th_ref
        scale = np.max(np.abs(y))
        out[k] = float(np.max(np.abs(x - y)) / scale) if scale > 0 else float(np.max(np.abs(x - y)))
    return out


def control_run(dycore, st0, nsteps):
    """States after 1..nsteps steps of the unperturbed run.
    Sec. 4.4: probtest-style ensemble verification, a reading."""
    out, st = [], st0
    for _ in range(nsteps):
        st = dycore.step(st)
        out.append(st)
    return out


def ensemble_spread(dycore, st0, eps, seeds, nsteps, control=None):
    """spread[field][n] = max over members of differences(member_n, control_n).
    Sec. 4.4: probtest-style ensemble verification, a reading."""
    if control is None:
        control = control_run(dycore, st0, nsteps)
    spread = {k: [0.0] * nsteps for k in FIELDS}
    for seed in seeds:
        st = perturb_state(st0, eps, seed)
        st["exner_pr"] = dycore.initial_exner_pr(st["exner"])
        for n in range(nsteps):
            st = dycore.step(st)
            d = differences(st, control[n], dycore)
            for k in FIELDS:
                spread[k][n] = max(spread[k][n], d[k])
    return spread
