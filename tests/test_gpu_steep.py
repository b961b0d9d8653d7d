"""Steep terrain on the GPU against the terrain oracle (oracle/terrain.py)
with its two steep-terrain options on: the pressure gradient at constant
height at the edge levels whose two cells' levels are offset by more than
half a layer, and the enhanced near-surface temperature diffusion.

A steep Gaussian mountain (3 km high, 400 km e-folding radius) on R2B3 with
30 levels, dt 600 s, 5 substeps, Rayleigh damping; the enhanced diffusion with
factor 0.2, threshold 1 K over the lowest 5 levels, so that it acts on the
mountain's flanks.  Parity after 1 step (1e-12) and 10 steps (1e-9), with the
probtest reading of Sec. 4.4 where a field's own conditioning is coarser;
the options change the result (both paths run); the mixed modes stay close to
the FP64 oracle; and the enhanced diffusion alone matches the oracle on a
near-surface spike over flat ground."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state, mountain_height, terrain_following_z
from oracle import Dycore as OracleDycore, DycoreParams, probtest
from oracle.terrain import TerrainDycore
from parity import gpu_params, to_torch, to_numpy, rel_err

pytestmark = pytest.mark.gpu

BIS, NLEV, DT = 3, 30, 600.0
STEEP = dict(steep_hpg=True, hdiff_tenh_fac=0.2, hdiff_tenh_thresh=1.0, hdiff_tenh_levels=5)


def _gpu_params(op, **over):
    d = gpu_params(op, steep_hpg=int(op.steep_hpg), hdiff_tenh_fac=op.hdiff_tenh_fac,
                   hdiff_tenh_thresh=op.hdiff_tenh_thresh, hdiff_tenh_levels=op.hdiff_tenh_levels)
    d.update(over)
    return d


@pytest.fixture(scope="module")
def steep():
    grid, z = make_grid(BIS), make_vct(NLEV)
    zz = terrain_following_z(z, mountain_height(grid.cell_xyz, h0=3000.0, d=4.0e5))
    op = DycoreParams(dtime=DT, ndyn_substeps=5, rayleigh_coeff=0.05, **STEEP)
    od = TerrainDycore(grid, zz, op)
    st = jw_type_state(grid, zz, seed=4)
    st["exner_pr"] = od.initial_exner_pr(st["exner"])
    states = [st]
    for _ in range(10):
        states.append(od.step(states[-1]))
    spread = probtest.ensemble_spread(od, st, 1e-16, (1, 2), 10, control=states[1:])
    return grid, zz, op, od, states, spread


def test_steep_terrain_steps_match_the_oracle(built_lib, cuda, steep):
    import paper_2608_21150_gb300 as P
    grid, zz, op, od, states, spread = steep
    assert od.v.steep["flag"].sum() > 50
    ex = od.enhanced_edge_factor(states[1]["theta_v"])
    assert np.count_nonzero(ex) > 10               # the enhanced diffusion acts
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, zz, _gpu_params(op))
    t = to_torch(states[0], cuda)
    errs = {}
    for n in range(1, 11):
        d.step(t)
        if n in (1, 10):
            errs[n] = rel_err(to_numpy(t), states[n], od)
    for n, base in ((1, 1e-12), (10, 1e-9)):
        tol = {k: max(base, 5.0 * spread[k][n - 1]) for k in spread}
        assert all(errs[n][k] < tol.get(k, base) for k in errs[n]), (n, errs[n], tol)


def test_the_steep_options_change_the_step(built_lib, cuda, steep):
    import paper_2608_21150_gb300 as P
    grid, zz, op, od, states, spread = steep
    g = P.Grid(grid, radius=op.radius)
    results = {}
    for name, over in (("both", {}), ("hpg", dict(hdiff_tenh_fac=0.0)), ("none", dict(steep_hpg=0, hdiff_tenh_fac=0.0))):
        d = P.Dycore(g, zz, _gpu_params(op, **over))
        t = to_torch(states[0], cuda)
        d.step(t)
        results[name] = to_numpy(t)
    assert np.max(np.abs(results["hpg"]["vn"] - results["none"]["vn"])) > 1e-6
    assert np.max(np.abs(results["both"]["theta_v"] - results["hpg"]["theta_v"])) > 1e-6


@pytest.mark.parametrize("prec", ["mixed", "f64col"])
def test_mixed_steep_terrain_close_to_the_fp64_oracle(built_lib, cuda, steep, prec):
    import paper_2608_21150_gb300 as P
    grid, zz, op, od, states, spread = steep
    g = P.Grid(grid, radius=op.radius)
    prec_id = P.ICON_PREC_MIXED if prec == "mixed" else P.ICON_PREC_MIXED_F64COL
    d = P.Dycore(g, zz, _gpu_params(op, precision=prec_id))
    t = to_torch(states[0], cuda)
    errs = {}
    for n in range(1, 11):
        d.step(t)
        if n in (1, 10):
            errs[n] = rel_err(to_numpy(t), states[n], od)
    assert all(e < 2e-5 for e in errs[1].values()), errs[1]
    assert all(e < 1e-3 for e in errs[10].values()), errs[10]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_enhanced_diffusion_on_a_near_surface_spike(built_lib, cuda, prec):
    """Flat R2B2: one diffusion call (icon_nh_diff) on a state with a 20 K
    spike in the lowest level of one cell equals the oracle's diffusion."""
    import paper_2608_21150_gb300 as P
    grid, z = make_grid(2), make_vct(20)
    op = DycoreParams(dtime=900.0, hdiff_tenh_fac=0.2, hdiff_tenh_thresh=5.0, hdiff_tenh_levels=4)
    od = OracleDycore(grid, z, op)
    st = jw_type_state(grid, z, seed=0)
    st["exner_pr"] = od.initial_exner_pr(st["exner"])
    st["theta_v"][37, -1] += 20.0
    ref = od.diffusion(st)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, _gpu_params(op, precision=P.ICON_PREC_MIXED if prec == "mixed" else P.ICON_PREC_FP64))
    t = to_torch(st, cuda)
    d.nh_diff(t)
    got = to_numpy(t)
    tol = 1e-12 if prec == "fp64" else 2e-5
    errs = rel_err(got, ref, od)
    assert all(e < tol for e in errs.values()), errs
    # the spike decayed more than the plain diffusion lets it
    plain = OracleDycore(grid, z, DycoreParams(dtime=900.0)).diffusion(st)
    assert got["theta_v"][37, -1] < plain["theta_v"][37, -1] - 0.5
