"""GPU diagnostics (ps, T850, mass, non-finite check) against the oracle's
definitions on the same state; a NaN injected on the host is reported as
ICON_ERR_NUMERIC without touching the GPU's health (no device fault)."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy
from oracle.diagnostics import surface_pressure, temperature_850, total_mass

pytestmark = pytest.mark.gpu


def test_diagnostics_match_oracle(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    t = to_torch(st, cuda)
    for _ in range(2):
        d.step(t)
    ps = torch.empty(grid.n_cells, dtype=torch.float64, device=cuda)
    t850 = torch.empty_like(ps)
    mass = d.diagnostics(t, ps, t850)
    s = to_numpy(t)
    ref_ps = surface_pressure(od, s["exner"], s["theta_v"])
    ref_t = temperature_850(od, s["exner"], s["theta_v"])
    assert np.max(np.abs(ps.cpu().numpy() - ref_ps) / ref_ps) < 1e-13
    assert np.max(np.abs(t850.cpu().numpy() - ref_t) / ref_t) < 1e-12
    assert abs(mass / total_mass(od, s["rho"]) - 1) < 1e-13
    assert np.allclose(g.cell_areas(), od.g.cell_area, rtol=1e-14, atol=0)


def test_non_finite_state_is_reported(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(1, 30, 1800.0)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, gpu_params(op))
    st["theta_v"][3, 7] = np.nan  # injected on the host
    t = to_torch(st, cuda)
    with pytest.raises(P.IconError) as e:
        d.diagnostics(t)
    assert e.value.code == P.ICON_ERR_NUMERIC
    st["theta_v"][3, 7] = 300.0
    st["vn"][5, 2] = np.inf
    t = to_torch(st, cuda)
    with pytest.raises(P.IconError) as e:
        d.diagnostics(t)
    assert e.value.code == P.ICON_ERR_NUMERIC
