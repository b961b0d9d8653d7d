"""Whole steps of a state in host memory: the library copies vn and w in, the
other four fields on a second stream while the first velocity tendencies run,
and rho and exner_pr back while the diffusion runs.  The result must be the
device-array step's, bit for bit: pinned and pageable host memory, with and
without the step's CUDA graph, FP64 and both mixed modes, and a substep of
host arrays (copied in and out in order) between the steps."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f64col"])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_host_array_steps_equal_device_steps(built_lib, cuda, precision, use_graph):
    import torch
    import paper_2608_21150_gb300 as P
    prec = {"fp64": P.ICON_PREC_FP64, "mixed": P.ICON_PREC_MIXED, "mixed_f64col": P.ICON_PREC_MIXED_F64COL}[precision]
    grid, z, op, od, st = setup(3, 30, 900.0, seed=6, rayleigh=0.05)
    g = P.Grid(grid, radius=op.radius)
    par = gpu_params(op, precision=prec, rayleigh_coeff=0.05, use_graph=use_graph, autotune=0, column_chunk=6)
    ref = P.Dycore(g, z, par)
    t = to_torch(st, cuda)
    for _ in range(3):
        ref.step(t)
    ref.nh_solve(t)
    ref.step(t)
    ref.synchronize()
    want = to_numpy(t)
    d = P.Dycore(g, z, par)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in st.items()}
    pageable = {k: np.ascontiguousarray(v).copy() for k, v in st.items()}
    for _ in range(3):
        d.step(pinned)
        d.step(pageable)
    d.nh_solve(pinned)
    d.nh_solve(pageable)
    d.step(pinned)
    d.step(pageable)
    for k in FIELDS:
        assert np.array_equal(pinned[k].numpy(), want[k]), ("pinned", k)
        assert np.array_equal(pageable[k], want[k]), ("pageable", k)
    ref.close()
    d.close()
