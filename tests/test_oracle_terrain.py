"""Pins of the terrain-following oracle (oracle/terrain.py) over the Gaussian
mountain of icon_inputs.terrain (2 km high, 1500 km e-folding radius).

* Flat ground: it reproduces the flat oracle (to the 1e-12 of one step).
* The per-column reference atmosphere stays at rest over the mountain, to
  rounding.
* Mass, sum A_c dz_c rho, is conserved exactly with flow over the mountain.
* A pressure perturbation that depends on height only exerts no horizontal
  force: along model levels its gradient is cancelled by the chain-rule
  term to rounding.
* The contravariant correction of a rigid rotation over the mountain converges
  to u . grad h (1 - z_flat/z_top), the vertical velocity of flow that follows
  the coordinate surfaces (measured 5.9 % RMS at R2B3, 2.8 % at R2B4), and a
  substep leaves w at the ground at that value (kinematic condition).
* Flow along the coordinate surfaces (w = w_concorr) has no vertical advection
  and is steady in the column solve; the per-column Rayleigh profile and the
  column solve over flat heights are the flat oracle's."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state, mountain_height, terrain_following_z
from oracle import Dycore, DycoreParams
from oracle.terrain import TerrainDycore
from parity import rel_err

A = 6.371229e6
U = 20.0


@pytest.fixture(scope="module")
def mountain3():
    grid, z = make_grid(3), make_vct(10)
    return grid, z, TerrainDycore(grid, terrain_following_z(z, mountain_height(grid.cell_xyz)), DycoreParams())


def _resting(t):
    th, ex = t.reference_state()
    p = t.p
    rho = p.p00 * ex ** (p.cvd / p.rd) / (p.rd * th)
    nlev = ex.shape[1]
    return dict(vn=np.zeros((t.g.ne, nlev)), w=np.zeros((t.g.nc, nlev + 1)), rho=rho, exner=ex.copy(),
                theta_v=th.copy(), exner_pr=np.zeros_like(ex))


def _rotation(t, nlev):
    u = U * np.cross([0.0, 0.0, 1.0], t.g.E)
    return np.repeat(np.sum(u * t.g.normal, 1)[:, None], nlev, 1)


def _u_dot_grad_h(t, h):
    """u . grad h at the cell centres for the rigid rotation and the Gaussian mountain."""
    lon, lat = np.deg2rad(90.0), np.deg2rad(30.0)
    centre = np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])
    x = t.g.C
    cx = x @ centre
    r = A * np.arccos(np.clip(cx, -1.0, 1.0))
    u = U * np.cross([0.0, 0.0, 1.0], x)
    # dh/dr = -2 r h / d^2, grad r = -(projected centre direction)/sin(angle)
    return (2.0 * r * h / 1.5e6 ** 2) * (u @ centre) / np.sqrt(1.0 - cx ** 2)


def test_flat_ground_reproduces_the_flat_oracle():
    grid, z = make_grid(2), make_vct(30)
    d = Dycore(grid, z, DycoreParams())
    st = jw_type_state(grid, z, seed=1)
    st["exner_pr"] = d.initial_exner_pr(st["exner"])
    t = TerrainDycore(grid, np.tile(z, (grid.n_cells, 1)), DycoreParams())
    errs = rel_err(t.step(st), d.step(st), d)
    assert max(errs.values()) < 1e-12, errs


def test_reference_atmosphere_over_the_mountain_stays_at_rest(mountain3):
    _, _, t = mountain3
    st = _resting(t)
    st["exner_pr"] = t.initial_exner_pr(st["exner"])
    assert np.all(st["exner_pr"] == 0.0)
    out = t.step(st)
    assert np.max(np.abs(out["vn"])) < 1e-12 and np.max(np.abs(out["w"])) < 1e-12
    assert np.max(np.abs(out["rho"] - st["rho"]) / st["rho"]) < 1e-14


def test_mass_is_conserved_over_the_mountain(mountain3):
    _, _, t = mountain3
    st = _resting(t)
    nlev = t.v.nlev
    st["vn"] = _rotation(t, nlev)
    st["w"] = t.w_concorr(st["vn"])
    st["theta_v"] = st["theta_v"] * (1.0 + 1e-3 * np.random.default_rng(0).standard_normal(st["theta_v"].shape))
    m0 = t.total_mass(st["rho"])
    out = t.step(st)
    assert all(np.all(np.isfinite(out[k])) for k in out)
    assert abs(t.total_mass(out["rho"]) - m0) / m0 < 1e-14
    assert np.max(np.abs(out["rho"] - st["rho"])) > 1e-8        # the flow did move mass around


def test_height_only_pressure_perturbation_exerts_no_horizontal_force(mountain3):
    _, _, t = mountain3
    pr = 1e-5 * t.v.z_mc
    theta_e = np.full((t.g.ne, t.v.nlev), 300.0)
    along_levels = t.p.cpd * 300.0 * t.grad_n(pr)
    hpg = t.horizontal_pressure_gradient(pr, theta_e)
    assert np.max(np.abs(along_levels)) > 1e-3
    assert np.max(np.abs(hpg)) < 1e-12 * np.max(np.abs(along_levels))


def test_contravariant_correction_and_kinematic_ground_condition(mountain3):
    grid, z, t = mountain3
    nlev = t.v.nlev
    h = mountain_height(grid.cell_xyz)
    vn = _rotation(t, nlev)
    ref = _u_dot_grad_h(t, h)
    wc = t.w_concorr(vn)
    assert np.all(wc[:, 0] == 0.0)                               # flat model top
    for k in (nlev, nlev // 2):
        lifted = ref * (1.0 - z[k] / z[0])
        err = np.sqrt(np.mean((wc[:, k] - lifted) ** 2)) / np.sqrt(np.mean(lifted ** 2))
        assert err < 0.1, (k, err)
    st = _resting(t)
    st["vn"], st["w"] = vn, wc
    out = t.substep(st)
    err = np.sqrt(np.mean((out["w"][:, nlev] - ref) ** 2)) / np.sqrt(np.mean(ref ** 2))
    assert err < 0.1, err


def test_rayleigh_profile_per_column_is_the_flat_one():
    """Every column's damping profile is the flat profile of its heights (the top
    is flat); over flat ground it equals the flat oracle's, which is pinned by
    its closed form."""
    grid, z = make_grid(1), make_vct(30)
    prm = DycoreParams(rayleigh_coeff=1.0 / 600.0, damp_height=10000.0)
    t = TerrainDycore(grid, np.tile(z, (grid.n_cells, 1)), prm)
    flat = Dycore(grid, z, prm).v.rayleigh_factor(120.0, prm)
    f = t.v.rayleigh_factor(120.0, prm)
    assert np.max(flat) > 0.1 and np.array_equal(f, np.tile(flat, (grid.n_cells, 1)))


def test_flow_along_the_coordinate_surfaces_has_no_vertical_advection(mountain3):
    """vn sheared in height, w = w_concorr(vn): the contravariant velocity is
    zero, so the vn tendency is the along-level part alone, which is the flat
    oracle's tendency at zero vertical velocity."""
    grid, z, t = mountain3
    nlev = t.v.nlev
    zc = 0.5 * (t.v.z_mc[t.g.e2c[:, 0]] + t.v.z_mc[t.g.e2c[:, 1]])
    vn = _rotation(t, nlev) * (1.0 + 1e-4 * zc)
    wc = t.w_concorr(vn)
    ddt_vn, ddt_w, _ = t.velocity_tendencies(vn, wc)
    assert ddt_vn.shape == (t.g.ne, nlev) and ddt_w.shape == (t.g.nc, nlev + 1)
    flat, _, _ = Dycore(grid, z, DycoreParams()).velocity_tendencies(vn, np.zeros_like(wc))
    assert np.max(np.abs(ddt_vn - flat)) < 1e-13 * np.max(np.abs(flat))


def test_flow_along_the_coordinate_surfaces_is_steady_in_the_column_solve(mountain3):
    """Reference atmosphere, w = w_concorr, no horizontal flux divergence and no
    advective tendency: nothing crosses the coordinate surfaces, so the column
    solve keeps w, rho and exner.  Without a w_concorr argument the solve over
    flat heights, Rayleigh damping included, is the flat oracle's."""
    grid, z, t = mountain3
    st = _resting(t)
    nlev = t.v.nlev
    wc = t.w_concorr(_rotation(t, nlev))
    st["w"] = wc.copy()
    v = t.v
    zero_c = np.zeros((t.g.nc, nlev))
    out = t.vertical_solve(st, v.interp_ic(st["rho"]), v.interp_ic(st["theta_v"]), v.interp_ic(zero_c),
                           zero_c, zero_c, np.zeros((t.g.nc, nlev + 1)), 120.0, wc)
    assert np.max(np.abs(out["w"] - wc)) < 1e-15 * np.max(np.abs(wc))
    assert np.max(np.abs(out["rho"] - st["rho"]) / st["rho"]) < 1e-15
    assert np.max(np.abs(out["exner"] - st["exner"])) < 1e-15
    damped = DycoreParams(rayleigh_coeff=1.0 / 600.0, damp_height=5000.0)
    d = Dycore(grid, z, damped)
    tf = TerrainDycore(grid, np.tile(z, (grid.n_cells, 1)), damped)
    s = jw_type_state(grid, z, seed=2)
    rng = np.random.default_rng(9)
    s["w"] = 0.05 * rng.standard_normal(s["w"].shape)
    s["w"][:, 0] = s["w"][:, -1] = 0.0
    args = (d.v.interp_ic(s["rho"]), d.v.interp_ic(s["theta_v"]), d.v.interp_ic(s["theta_v"] - d.v.theta_ref),
            1e-6 * rng.standard_normal((grid.n_cells, nlev)), 1e-4 * rng.standard_normal((grid.n_cells, nlev)),
            1e-3 * rng.standard_normal((grid.n_cells, nlev + 1)), 120.0)
    a, b = d.vertical_solve(s, *args), tf.vertical_solve(s, *args)
    for k in ("w", "rho", "exner", "theta_v"):
        assert np.array_equal(a[k], b[k]), k


def test_pressure_gradient_error_over_the_mountain_converges_at_second_order():
    """Resting isothermal atmosphere (260 K, not the reference state) over the
    mountain: its pressure depends on height only, so the true horizontal force
    is zero.  Along model levels the gradient of the exner perturbation is
    large; the chain-rule term cancels it up to the error of the centred
    vertical difference, second order in the layer thickness (measured ratios
    4.16, 4.08 per halving; 0.9 % of the along-level gradient at 60 levels)."""
    grid = make_grid(3)
    h = mountain_height(grid.cell_xyz)
    p, T = DycoreParams(), 260.0
    errs = []
    for nlev in (15, 30, 60):
        t = TerrainDycore(grid, terrain_following_z(make_vct(nlev, dz_sfc=30000.0 / nlev / 4), h), p)
        pi = np.exp(-p.grav * t.v.z_mc / (p.cpd * T))
        th = T / pi
        th_e = 0.5 * (th[t.g.e2c[:, 0]] + th[t.g.e2c[:, 1]])
        pr = pi - t.v.exner_ref
        errs.append(np.max(np.abs(t.horizontal_pressure_gradient(pr, th_e))))
        along = np.max(np.abs(p.cpd * th_e * t.grad_n(pr)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 0.02 * along


def test_diagnostics_use_each_columns_ground(mountain3):
    """Surface pressure over the mountain: the resting reference atmosphere
    extrapolated from its lowest level to its own ground matches the
    continuous reference p00 exp(-z_sfc/H)^(cpd/rd) to the discretisation
    error (1e-4); the mass diagnostic sums each column's own layers."""
    from oracle import diagnostics
    grid, z, t = mountain3
    st = _resting(t)
    p = t.p
    ps = diagnostics.surface_pressure(t, st["exner"], st["theta_v"])
    z_sfc = t.v.z_ifc[:, -1]
    assert z_sfc.max() > 1500.0
    H = p.cpd * p.ref_T0 / p.grav
    exact = p.p00 * np.exp(-z_sfc / H) ** (p.cpd / p.rd)
    assert np.max(np.abs(ps / exact - 1.0)) < 1e-4
    assert diagnostics.total_mass(t, st["rho"]) == t.total_mass(st["rho"])


def test_corrector_features_use_each_columns_reference(mountain3):
    """The corrector's exner and theta_v features are deviations from the
    cell's own reference column: zero for the resting reference atmosphere."""
    from oracle import corrector
    grid, z, t = mountain3
    st = _resting(t)
    x = corrector.column_features(t, st)
    nlev = st["exner"].shape[1]
    assert x.shape == (grid.n_cells, 5 * nlev)
    assert np.all(x[:, nlev:3 * nlev] == 0.0)


# ---------------------------------------------------------------------------
# steep terrain: the constant-height pressure gradient and the enhanced
# near-surface temperature diffusion

@pytest.fixture(scope="module")
def steep3():
    """A steep Gaussian mountain, 3 km high with a 400 km e-folding radius, on
    R2B3 with 30 levels: the lowest levels of neighbouring columns are offset
    by more than half a layer near its flanks."""
    grid, z = make_grid(3), make_vct(30)
    h = mountain_height(grid.cell_xyz, h0=3000.0, d=4.0e5)
    return grid, z, h, TerrainDycore(grid, terrain_following_z(z, h), DycoreParams(steep_hpg=True))


def test_constant_height_weights_reproduce_quadratics_and_flag_only_offset_levels(steep3):
    grid, z, h, t = steep3
    st = t.v.steep
    assert 50 < st["flag"].sum() < 0.2 * st["flag"].size
    z_e = st["z_e"]
    for s in (0, 1):
        zc = t.v.z_mc[t.g.e2c[:, s]]
        w, k0 = st["w_%d" % s], st["k0_%d" % s]
        zj = np.stack([np.take_along_axis(zc, k0 + j, axis=1) for j in range(3)], axis=-1)
        assert np.max(np.abs(w.sum(-1) - 1.0)) < 1e-12
        assert np.max(np.abs((w * zj).sum(-1) - z_e)) < 1e-9 * 3e4
        assert np.max(np.abs((w * zj ** 2).sum(-1) - z_e ** 2)) < 1e-9 * 9e8
    flat = TerrainDycore(grid, np.tile(z, (grid.n_cells, 1)), DycoreParams(steep_hpg=True))
    assert not flat.v.steep["flag"].any()


def _isothermal(t, T=260.0):
    p = t.p
    pi = np.exp(-p.grav * t.v.z_mc / (p.cpd * T))
    th = T / pi
    return pi, th, 0.5 * (th[t.g.e2c[:, 0]] + th[t.g.e2c[:, 1]])


def test_constant_height_gradient_is_exact_for_exner_quadratic_in_height(steep3):
    """A total exner quadratic in height exerts no horizontal force; the
    constant-height form sees none at the steep points (the Lagrange
    quadratic reproduces it), the chain-rule form does."""
    grid, z, h, t = steep3
    zm = t.v.z_mc
    pi = 1.0 - 1.1e-4 * zm + 3.0e-9 * zm ** 2
    th_e = np.full((t.g.ne, t.v.nlev), 300.0)
    pr = pi - t.v.exner_ref
    along = t.p.cpd * th_e * t.grad_n(pr)
    fl = t.v.steep["flag"]
    hpg = t.horizontal_pressure_gradient(pr, th_e)
    chain = TerrainDycore(grid, t.v.z_ifc, DycoreParams()).horizontal_pressure_gradient(pr, th_e)
    scale = np.max(np.abs(along[fl]))
    assert np.max(np.abs(hpg[fl])) < 1e-9 * scale
    assert np.max(np.abs(chain[fl])) > 1e-4 * scale
    # elsewhere the two forms are the same
    assert np.array_equal(hpg[~fl], chain[~fl])


def test_constant_height_gradient_beats_the_chain_rule_at_steep_points():
    """Resting isothermal atmosphere (not the reference state) over a steeper
    mountain (3 km, 300 km) on R2B4: where the edge height lies between the
    levels of both neighbour columns, the constant-height form's spurious
    force is below a quarter of the chain-rule form's at 15, 30 and 60 levels
    (measured 0.07, 0.13, 0.16)."""
    grid = make_grid(4)
    h = mountain_height(grid.cell_xyz, h0=3000.0, d=3.0e5)
    for nlev in (15, 30, 60):
        zz = terrain_following_z(make_vct(nlev, dz_sfc=30000.0 / nlev / 4), h)
        t = TerrainDycore(grid, zz, DycoreParams(steep_hpg=True))
        c = TerrainDycore(grid, zz, DycoreParams())
        pi, th, th_e = _isothermal(t)
        pr = pi - t.v.exner_ref
        st = t.v.steep
        inside = st["flag"].copy()
        for s in (0, 1):
            zc = t.v.z_mc[t.g.e2c[:, s]]
            lo = np.take_along_axis(zc, st["k0_%d" % s] + 2, axis=1)
            hi = np.take_along_axis(zc, st["k0_%d" % s], axis=1)
            inside &= (st["z_e"] >= lo) & (st["z_e"] <= hi)
        assert inside.sum() > 20
        e_const = np.max(np.abs(t.horizontal_pressure_gradient(pr, th_e)[inside]))
        e_chain = np.max(np.abs(c.horizontal_pressure_gradient(pr, th_e)[inside]))
        assert e_const < 0.25 * e_chain, (nlev, e_const, e_chain)


def _spiked(seed=0, k_spike=None, amp=20.0):
    grid, z = make_grid(2), make_vct(20)
    p = DycoreParams(dtime=900.0, hdiff_tenh_fac=0.2, hdiff_tenh_thresh=5.0, hdiff_tenh_levels=4)
    d = Dycore(grid, z, p)
    st = jw_type_state(grid, z, seed=seed)
    st["exner_pr"] = d.initial_exner_pr(st["exner"])
    k = d.v.nlev - 1 if k_spike is None else k_spike
    c = 37
    st["theta_v"] = st["theta_v"].copy()
    st["theta_v"][c, k] += amp
    return grid, z, p, d, st, c, k


def test_enhanced_temperature_diffusion_is_off_below_the_threshold():
    grid, z = make_grid(2), make_vct(20)
    st = jw_type_state(grid, z, seed=1)
    on = Dycore(grid, z, DycoreParams(dtime=900.0, hdiff_tenh_fac=0.2))
    off = Dycore(grid, z, DycoreParams(dtime=900.0))
    st["exner_pr"] = on.initial_exner_pr(st["exner"])
    th = st["theta_v"]
    g = on.g
    nbr = (th[g.c2e2c[:, 0]] + th[g.c2e2c[:, 1]] + th[g.c2e2c[:, 2]]) / 3.0
    assert np.max(np.abs(th - nbr)[:, -5:]) < 5.0        # no cell above the threshold in the lowest levels
    a, b = on.diffusion(st), off.diffusion(st)
    for k in ("theta_v", "exner", "vn", "w"):
        assert np.array_equal(a[k], b[k]), k


def test_enhanced_temperature_diffusion_acts_on_a_near_surface_spike_only():
    """A 20 K spike in the lowest level of one cell: the enhanced flux acts on
    that level only, within two rings of cells (the spike's neighbours differ
    from their own neighbours' mean by about 20/3 K, above the threshold too),
    and adds exactly the closed-form change
    dt/A_c sum_e l_e/d_e (0.2 A_e/dt) (theta_nbr - theta_c) at the spike (its
    excess factor is 1: 20 K - 5 K > 5 K), keeps sum A theta, and does nothing
    for the same spike at the model top."""
    grid, z, p, d, st, c, k = _spiked()
    off = Dycore(grid, z, DycoreParams(dtime=900.0))
    a, b = d.diffusion(st), off.diffusion(st)
    diff = a["theta_v"] - b["theta_v"]
    changed = np.argwhere(diff != 0.0)
    g = d.g
    ring1 = {c} | set(g.c2e2c[c].tolist())
    ring2 = set(ring1)
    for n in ring1:
        ring2 |= set(g.c2e2c[n].tolist())
    assert set(changed[:, 0].tolist()) <= ring2 and set(changed[:, 1].tolist()) == {k}
    assert ring1 <= set(changed[:, 0].tolist())
    th = st["theta_v"]
    closed = 0.0
    for j in range(3):
        e = g.c2e[c, j]
        closed += g.edge_length[e] / g.dual_length[e] * (0.2 * g.edge_area[e] / p.dtime) \
            * (th[g.c2e2c[c, j], k] - th[c, k])
    closed *= p.dtime / g.cell_area[c]
    assert abs(diff[c, k] - closed) < 1e-10 * abs(closed)
    area = g.cell_area[:, None]
    assert abs(np.sum(area * a["theta_v"]) / np.sum(area * th) - 1.0) < 1e-14
    _, _, _, d0, st0, c0, k0 = _spiked(k_spike=0)
    assert np.array_equal(d0.diffusion(st0)["theta_v"], off.diffusion(st0)["theta_v"])
