"""The fused velocity-advection kernel (rows A1-A4 in one launch over patches
of 128 consecutive cells, intermediates in shared memory) against the four
separate kernels: the same expressions in the same order, so whole mixed-
precision steps must agree bit for bit.  Grids: R2B0 (one patch larger than
the grid), R2B1 (a ragged last patch of 64 cells), R2B4 (160 patches, levels
not a multiple of the 8-level chunk)."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")


@pytest.mark.parametrize("bisections,nlev", [(0, 2), (1, 9), (4, 30)])
@pytest.mark.parametrize("precision", ["mixed", "mixed_f64col"])
def test_fused_advection_matches_the_four_kernels_bitwise(built_lib, cuda, bisections, nlev, precision):
    import paper_2608_21150_gb300 as P
    prec = P.ICON_PREC_MIXED if precision == "mixed" else P.ICON_PREC_MIXED_F64COL
    grid, z, op, od, st = setup(bisections, nlev, 720.0, seed=5, rayleigh=0.05)
    g = P.Grid(grid, radius=op.radius)
    runs = []
    for fused in (1, 0):
        # the same launch shapes for both (no autotuning), so that only rows A1-A4 differ
        d = P.Dycore(g, z, gpu_params(op, precision=prec, rayleigh_coeff=0.05, fused_advection=fused,
                                      autotune=0, column_chunk=6))
        t = to_torch(st, cuda)
        for _ in range(3):
            d.step(t)
        d.synchronize()
        runs.append(to_numpy(t))
        d.close()
    for k in FIELDS:
        assert np.all(np.isfinite(runs[0][k])), k
        assert np.array_equal(runs[0][k], runs[1][k]), (k, float(np.max(np.abs(runs[0][k] - runs[1][k]))))
