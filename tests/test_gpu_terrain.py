"""The terrain-following dycore on the GPU (icon_dycore_create_terrain)
against the terrain oracle (oracle/terrain.py), over the Gaussian mountain of
the mountain configuration (2 km high, 1500 km e-folding radius, centred at
90E 30N) on R2B2 with 30 levels, dt 1800 s, 5 substeps, Rayleigh damping:

* whole-step parity after 1 step (1e-12) and 10 steps (1e-9), with the
  probtest reading of Sec. 4.4 (five times the oracle's spread under
  rounding-level input perturbations) where a field's own conditioning is
  coarser than the gate;
* equal columns (flat heights given per column) step bit for bit like the
  flat dycore, FP64 and mixed (the mixed mode with an FP64 column solve to
  rounding);
* the per-column reference atmosphere stays at rest over the mountain;
* the total mass is conserved; the diagnostics and the corrector's features
  use each column's ground and reference state;
* the mixed mode over terrain stays close to the FP64 oracle;
* invalid heights are refused and the per-level reference query says why."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state, mountain_height, terrain_following_z
from oracle import DycoreParams, probtest
from oracle import corrector as oc
from oracle.diagnostics import surface_pressure, temperature_850, total_mass
from oracle.terrain import TerrainDycore
from parity import gpu_params, to_torch, to_numpy, rel_err

pytestmark = pytest.mark.gpu

BIS, NLEV, DT, SEED = 2, 30, 1800.0, 3


@pytest.fixture(scope="module")
def mountain():
    grid, z = make_grid(BIS), make_vct(NLEV)
    zz = terrain_following_z(z, mountain_height(grid.cell_xyz))
    op = DycoreParams(dtime=DT, ndyn_substeps=5, rayleigh_coeff=0.05)
    od = TerrainDycore(grid, zz, op)
    st = jw_type_state(grid, zz, seed=SEED)
    st["exner_pr"] = od.initial_exner_pr(st["exner"])
    states = [st]
    for _ in range(10):
        states.append(od.step(states[-1]))
    spread = probtest.ensemble_spread(od, st, 1e-16, (1, 2), 10, control=states[1:])
    return grid, z, zz, op, od, states, spread


def _gate(base, spread, n):
    return {k: max(base, 5.0 * spread[k][n - 1]) for k in spread}


@pytest.mark.parametrize("use_graph", [1, 0], ids=["graph", "direct"])
def test_terrain_steps_match_the_oracle(built_lib, cuda, mountain, use_graph):
    import paper_2608_21150_gb300 as P
    grid, z, zz, op, od, states, spread = mountain
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, zz, gpu_params(op, use_graph=use_graph))
    t = to_torch(states[0], cuda)
    errs = {}
    for n in range(1, 11):
        d.step(t)
        if n in (1, 10):
            errs[n] = rel_err(to_numpy(t), states[n], od)
    d.close()
    g.close()
    for n, base in ((1, 1e-12), (10, 1e-9)):
        tol = _gate(base, spread, n)
        assert all(errs[n][k] < tol.get(k, base) for k in errs[n]), (n, errs[n], tol)
    # the ground's w is the contravariant correction: nonzero over the slopes
    assert np.max(np.abs(states[10]["w"][:, -1])) > 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed", "f64col"])
def test_equal_columns_step_like_the_flat_dycore_bitwise(built_lib, cuda, prec):
    import paper_2608_21150_gb300 as P
    grid, z = make_grid(BIS), make_vct(NLEV)
    st = jw_type_state(grid, z, seed=SEED)
    op = DycoreParams(dtime=DT, ndyn_substeps=5, rayleigh_coeff=0.05)
    g = P.Grid(grid, radius=op.radius)
    prec_id = {"fp64": P.ICON_PREC_FP64, "mixed": P.ICON_PREC_MIXED, "f64col": P.ICON_PREC_MIXED_F64COL}[prec]
    params = gpu_params(op, precision=prec_id)
    flat = P.Dycore(g, z, params)
    terr = P.Dycore(g, np.tile(z, (grid.n_cells, 1)), params)
    st["exner_pr"] = st["exner"] - flat.reference_state()[1][None, :]
    a, b = to_torch(st, cuda), to_torch(st, cuda)
    for _ in range(2):
        flat.step(a)
        terr.step(b)
    for k in a:
        if prec == "f64col":
            # this mode's FP64 solve of FP32 inputs: the compiler fuses some
            # multiply-adds of the terrain form differently at one chunk
            # length, so equal columns agree to rounding, not bit for bit:
            # 1e-13 of each field, and for w (the residual of vertical forces
            # of order g dt_s, some 1e3 m/s) 1e-12 m/s
            scale = float(a[k].abs().max())
            tol = 1e-12 if k == "w" else 1e-13 * scale
            assert float((a[k] - b[k]).abs().max()) <= tol, k
        else:
            assert bool((a[k] == b[k]).all()), k
    th, ex = terr.reference_columns()
    th0, ex0 = flat.reference_state()
    assert np.array_equal(th, np.tile(th0, (grid.n_cells, 1))) and np.array_equal(ex, np.tile(ex0, (grid.n_cells, 1)))


def _resting(d, grid, op):
    th, ex = d.reference_columns()
    rho = op.p00 * ex ** (op.cvd / op.rd) / (op.rd * th)
    return dict(vn=np.zeros((grid.n_edges, NLEV)), w=np.zeros((grid.n_cells, NLEV + 1)), rho=rho, exner=ex.copy(),
                theta_v=th.copy(), exner_pr=np.zeros_like(ex))


def test_reference_atmosphere_over_the_mountain_stays_at_rest(built_lib, cuda, mountain):
    import paper_2608_21150_gb300 as P
    grid, z, zz, op, od, states, spread = mountain
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, zz, gpu_params(op))
    th, ex = d.reference_columns()
    th_o, ex_o = od.reference_state()
    assert np.max(np.abs(th - th_o) / th_o) < 1e-14 and np.max(np.abs(ex - ex_o) / ex_o) < 1e-14
    st = _resting(d, grid, op)
    t = to_torch(st, cuda)
    for _ in range(10):
        d.step(t)
    s = to_numpy(t)
    assert np.max(np.abs(s["vn"])) < 1e-12 and np.max(np.abs(s["w"])) < 1e-12
    assert np.max(np.abs(s["rho"] - st["rho"]) / st["rho"]) < 1e-13


def test_mass_and_diagnostics_over_the_mountain(built_lib, cuda, mountain):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, zz, op, od, states, spread = mountain
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, zz, gpu_params(op))
    t = to_torch(states[0], cuda)
    m0 = d.diagnostics(t)
    assert abs(m0 / total_mass(od, states[0]["rho"]) - 1.0) < 1e-14
    for _ in range(10):
        d.step(t)
    ps = torch.empty(grid.n_cells, dtype=torch.float64, device=cuda)
    t850 = torch.empty_like(ps)
    m1 = d.diagnostics(t, ps, t850)
    assert abs(m1 - m0) / m0 < 1e-13
    s = to_numpy(t)
    ref_ps = surface_pressure(od, s["exner"], s["theta_v"])
    ref_t = temperature_850(od, s["exner"], s["theta_v"])
    assert np.max(np.abs(ps.cpu().numpy() - ref_ps) / ref_ps) < 1e-13
    assert np.max(np.abs(t850.cpu().numpy() - ref_t) / ref_t) < 1e-12


@pytest.mark.parametrize("prec", ["mixed", "f64col"])
def test_mixed_over_terrain_close_to_the_fp64_oracle(built_lib, cuda, mountain, prec):
    import paper_2608_21150_gb300 as P
    grid, z, zz, op, od, states, spread = mountain
    g = P.Grid(grid, radius=op.radius)
    prec_id = P.ICON_PREC_MIXED if prec == "mixed" else P.ICON_PREC_MIXED_F64COL
    d = P.Dycore(g, zz, gpu_params(op, precision=prec_id))
    t = to_torch(states[0], cuda)
    errs = {}
    for n in range(1, 11):
        d.step(t)
        if n in (1, 10):
            errs[n] = rel_err(to_numpy(t), states[n], od)
    assert all(e < 2e-5 for e in errs[1].values()), errs[1]
    assert all(e < 1e-3 for e in errs[10].values()), errs[10]


def test_corrector_features_over_terrain(built_lib, cuda, mountain):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, zz, op, od, states, spread = mountain
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, zz, gpu_params(op))
    st = states[2]
    t = to_torch(st, cuda)
    cx = torch.empty((grid.n_cells, 5 * NLEV), dtype=torch.float32, device=cuda)
    ex = torch.empty((grid.n_edges, 11 * NLEV), dtype=torch.float32, device=cuda)
    d.corrector_features(t, cx, ex)
    d.synchronize()
    ocx = oc.column_features(od, st)
    got = cx.cpu().numpy().astype(np.float64)
    for j, sj in enumerate([0, 1, 2, 3, 3]):
        blk = slice(j * NLEV, (j + 1) * NLEV)
        scale = np.max(np.abs(ocx[:, sj * NLEV:(sj + 1) * NLEV]))
        assert np.max(np.abs(got[:, blk] - ocx[:, blk])) / scale < 2e-6, j


def test_invalid_heights_are_refused(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    grid, z = make_grid(1), make_vct(10)
    g = P.Grid(grid)
    zz = terrain_following_z(z, mountain_height(grid.cell_xyz))
    bad = zz.copy()
    bad[3, 4], bad[3, 5] = bad[3, 5], bad[3, 4]          # not decreasing
    with pytest.raises(P.IconError) as e:
        P.Dycore(g, bad, dict(dtime=900.0))
    assert e.value.code == P.ICON_ERR_ARG and b"decrease" in str(e.value).encode()
    bad = zz.copy()
    bad[7, 0] += 10.0                                    # a different model top
    with pytest.raises(P.IconError) as e:
        P.Dycore(g, bad, dict(dtime=900.0))
    assert e.value.code == P.ICON_ERR_ARG and b"top" in str(e.value).encode()
    d = P.Dycore(g, zz, dict(dtime=900.0))
    with pytest.raises(P.IconError) as e:
        d.reference_state()
    assert e.value.code == P.ICON_ERR_UNSUPPORTED
