"""Bitwise run-to-run determinism of the step (no atomics or order-dependent
reductions in the stencils or the column solve): the same input stepped twice
by one dycore, and once more by a second dycore whose launch shapes were
autotuned on its own, gives the same bits, in FP64 and in both mixed modes."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f64col"])
def test_repeated_steps_are_bitwise_identical(built_lib, cuda, precision):
    import paper_2608_21150_gb300 as P
    prec = {"fp64": P.ICON_PREC_FP64, "mixed": P.ICON_PREC_MIXED, "mixed_f64col": P.ICON_PREC_MIXED_F64COL}[precision]
    grid, z, op, od, st = setup(4, 30, 720.0, seed=3, rayleigh=0.05)
    g = P.Grid(grid, radius=op.radius)
    runs = []
    dycores = [P.Dycore(g, z, gpu_params(op, precision=prec, rayleigh_coeff=0.05)) for _ in range(2)]
    for d in (dycores[0], dycores[0], dycores[1]):
        t = to_torch(st, cuda)
        for _ in range(3):
            d.step(t)
        d.synchronize()
        runs.append(to_numpy(t))
    for r in runs[1:]:
        for k in FIELDS:
            assert np.array_equal(r[k], runs[0][k]), (precision, k)
    assert all(np.all(np.isfinite(runs[0][k])) for k in FIELDS)
    for d in dycores:
        d.close()
