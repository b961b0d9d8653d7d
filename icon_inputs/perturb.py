"""Seeded relative perturbations of an initial state (probtest ensembles).

Each perturbed field is multiplied point by point by (1 + eps u), u drawn
uniformly from [-1, 1) by numpy's PCG64 generator seeded with `seed`, fields
in the fixed order of `fields`.  Input generation only: no dynamics.
"""
import numpy as np

PERTURBED = ("vn", "rho", "exner", "theta_v")


def perturb_state(st, eps, seed, fields=PERTURBED):
    """A copy of the state dict with `fields` perturbed; other fields copied."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {k: np.array(v, dtype=np.float64, copy=True) for k, v in st.items()}
    for k in fields:
        u = rng.uniform(-1.0, 1.0, size=out[k].shape)
        out[k] *= 1.0 + eps * u
    return out
