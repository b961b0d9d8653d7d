"""Degenerate and empty inputs at the C-ABI.  The smallest problem the
library accepts (R2B0: 80 cells, 2 levels) steps like the oracle and keeps its
mass; empty or malformed requests are refused with ICON_ERR_ARG before any
memory is touched: zero columns or out-of-range level counts for the
allocation-free column solve, a vertical grid that does not decrease to a
flat ground, a non-positive time step or substep count, an unknown precision,
a NULL or mixed host/device state, and an MLP batch of zero or above the
network's maximum."""
import ctypes

import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy, rel_err

pytestmark = pytest.mark.gpu


def test_smallest_grid_steps_like_the_oracle(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(0, 2, 1800.0, seed=1)
    assert grid.n_cells == 80 and z.size == 3
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    t = to_torch(st, cuda)
    m0 = d.diagnostics(t)
    d.step(t)
    d.synchronize()
    errs = rel_err(to_numpy(t), od.step(st), od)
    assert max(errs.values()) < 1e-12, errs
    assert abs(d.diagnostics(t) - m0) / m0 < 1e-13
    d.close()


def _dycore_error(P, g, z, **over):
    with pytest.raises(P.IconError) as e:
        P.Dycore(g, z, P.default_params(**over))
    return e.value


def test_dycore_create_refuses_malformed_requests(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(1, 4, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    for zz, over in ((np.array([100.0, 0.0]), {}),                 # one level
                     (z[::-1].copy(), {}),                         # increasing heights
                     (z + 10.0, {}),                               # ground not at 0
                     (z, {"dtime": 0.0}), (z, {"ndyn_substeps": 0}),
                     (z, {"precision": 7}), (z, {"column_chunk": 3})):
        err = _dycore_error(P, g, zz, **over)
        assert err.code == P.ICON_ERR_ARG, (over, err)


def test_step_refuses_null_and_mixed_states(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(1, 4, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    t = to_torch(st, cuda)
    s = d._state(t)
    s.rho = None
    assert P.icon_dycore_step(d.handle, ctypes.byref(s)) == P.ICON_ERR_ARG
    mixed = dict(t)
    mixed["rho"] = np.ascontiguousarray(st["rho"])               # one host field among device fields
    s = d._state(mixed)
    assert P.icon_dycore_step(d.handle, ctypes.byref(s)) == P.ICON_ERR_ARG
    assert b"mixes host and device" in P.icon_last_error()
    d.close()


def test_noalloc_refuses_empty_and_out_of_range_sizes(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    x = torch.zeros(8, dtype=torch.float64, device=cuda)
    p = P.default_params()
    for n_cols, nlev in ((0, 30), (-1, 30), (10, 1), (10, 257)):
        z = np.ascontiguousarray(np.linspace(30000.0, 0.0, max(nlev, 1) + 1))
        rc = P.icon_column_solve_noalloc(n_cols, nlev, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(p), *([x.data_ptr()] * 4), None, None, x.data_ptr(), None,
                                         *([x.data_ptr()] * 6))
        assert rc == P.ICON_ERR_ARG, (n_cols, nlev)


def test_mlp_refuses_empty_and_oversized_batches(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    h = ctypes.c_void_p()
    assert P.icon_mlp_create(8, 64, 4, 100, ctypes.byref(h)) == P.ICON_ERR_ARG     # max_batch not a multiple of 64
    net = P.MLP(8, 64, 4, 128)
    x = torch.zeros((256, 8), dtype=torch.float32, device=cuda)
    y = torch.zeros((256, 4), dtype=torch.float32, device=cuda)
    for batch in (0, -5, 129):
        rc = P.icon_mlp_forward(net.handle, x.data_ptr(), batch, y.data_ptr(), None)
        assert rc == P.ICON_ERR_ARG, batch
    net.close()
