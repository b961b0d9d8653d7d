"""Stretched height-based vertical grid (flat ground).

Layer thicknesses grow geometrically from ``dz_sfc`` at the surface,
dz_j = dz_sfc * r**j (j = 0 at the surface), with r chosen so that the
layers sum to ``top``.  Half-level heights are returned top first:
z_ifc[0] = top, z_ifc[nlev] = 0, which is the level order of the fields
(k = 0 is the model top).
"""
import numpy as np


def stretch_ratio(nlev: int, top: float = 30000.0, dz_sfc: float = 50.0) -> float:
    """Solve sum_{j<nlev} dz_sfc*r**j = top for r > 1 by bisection."""
    if dz_sfc * nlev >= top:
        raise ValueError("uniform layers already exceed the top")
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        s = dz_sfc * (mid ** nlev - 1.0) / (mid - 1.0)
        if s > top:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def make_vct(nlev: int, top: float = 30000.0, dz_sfc: float = 50.0) -> np.ndarray:
    """Half-level heights [nlev+1], float64, top first."""
    r = stretch_ratio(nlev, top, dz_sfc)
    dz = dz_sfc * r ** np.arange(nlev)            # surface first
    z_up = np.concatenate([[0.0], np.cumsum(dz)])  # surface first
    z_up[-1] = top                                 # remove the bisection residue
    return np.ascontiguousarray(z_up[::-1], dtype=np.float64)
