"""Helpers shared by the GPU parity tests: run the same seeded inputs through
the oracle (CPU, FP64) and through the C-ABI library, and compare."""
import numpy as np

from icon_inputs import make_grid, make_vct, jw_type_state
from oracle import Dycore as OracleDycore, DycoreParams

PARAM_KEYS = ("dtime", "ndyn_substeps", "rayleigh_coeff", "damp_height", "divdamp_fac", "divflux_fac", "hdiff_temp")


def setup(bisections, nlev, dtime, seed=0, ndyn=5, rayleigh=0.0, **extra):
    grid = make_grid(bisections)
    z = make_vct(nlev)
    op = DycoreParams(dtime=dtime, ndyn_substeps=ndyn, rayleigh_coeff=rayleigh, **extra)
    od = OracleDycore(grid, z, op)
    st = jw_type_state(grid, z, seed=seed)
    st["exner_pr"] = od.initial_exner_pr(st["exner"])
    return grid, z, op, od, st


def gpu_params(op, **over):
    d = dict(dtime=op.dtime, ndyn_substeps=op.ndyn_substeps, rayleigh_coeff=op.rayleigh_coeff,
             damp_height=op.damp_height, divdamp_fac=op.divdamp_fac, divflux_fac=op.divflux_fac,
             hdiff_temp=int(op.hdiff_temp),
             vwind_impl_wgt=op.vwind_impl_wgt, exner_exfac=op.exner_exfac, hdiff_smag_fac=op.hdiff_smag_fac,
             hdiff_k4=op.hdiff_k4, hdiff_w_k4=op.hdiff_w_k4, ref_T0=op.ref_T0)
    d.update(over)
    return d


def to_torch(st, device):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in st.items()}


def to_numpy(st):
    return {k: v.detach().cpu().numpy() for k, v in st.items()}


def rel_err(gpu, ref, od):
    """Per-field relative inf-norm error; exner and theta_v as deviations from the
    oracle's reference profiles; exner_pr as is."""
    out = {}
    th_ref, ex_ref = od.reference_state()
    if ex_ref.ndim == 1:      # per column over terrain
        th_ref, ex_ref = th_ref[None, :], ex_ref[None, :]
    for k in ref:
        a, b = np.asarray(gpu[k]), np.asarray(ref[k])
        if k == "exner":
            a, b = a - ex_ref, b - ex_ref
        if k == "theta_v":
            a, b = a - th_ref, b - th_ref
        scale = np.max(np.abs(b))
        out[k] = float(np.max(np.abs(a - b)) / scale) if scale > 0 else float(np.max(np.abs(a - b)))
    return out
