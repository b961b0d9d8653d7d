"""Pins of the learned corrector's CPU oracle (oracle/corrector.py): the
features, targets, increments and check are fixed by closed forms and
invariants, independently of the oracle's own code path."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state
from oracle import Dycore, DycoreParams
from oracle import corrector as oc
from oracle import mlp as omlp


def _dycore(bis, nlev, ndyn=5, dtime=600.0):
    return Dycore(make_grid(bis), make_vct(nlev), DycoreParams(dtime=dtime, ndyn_substeps=ndyn))


def _solid_body(d, U, nlev):
    """vn of the zonal flow u = U cos(lat) east (vn = u . n_e at the edge midpoints)."""
    g = d.g
    east, _ = oc.east_north(g.E)
    coslat = np.sqrt(g.E[:, 0] ** 2 + g.E[:, 1] ** 2)
    vn = U * coslat * np.einsum("ex,ex->e", east, g.normal)
    return np.repeat(vn[:, None], nlev, axis=1)


def test_east_north_frame_at_closed_form_points():
    C = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [np.sqrt(0.5), 0.0, np.sqrt(0.5)]])
    east, north = oc.east_north(C)
    np.testing.assert_allclose(east, [[0, 1, 0], [-1, 0, 0], [0, 1, 0]], atol=1e-15)
    np.testing.assert_allclose(north, [[0, 0, 1], [0, 0, 1], [-np.sqrt(0.5), 0, np.sqrt(0.5)]], atol=1e-15)


def test_velocity_features_of_solid_body_rotation_converge():
    """u -> U cos(lat), v -> 0 at the cell centres, with the error falling at
    second order: the error falls about fourfold per bisection (Perot reconstruction of a smooth field)."""
    U, errs = 20.0, []
    for bis in (2, 3, 4):
        d = _dycore(bis, 2)
        g = d.g
        st = {"vn": _solid_body(d, U, 2), "w": np.zeros((g.nc, 3)),
              "exner": np.ones((g.nc, 2)), "theta_v": np.full((g.nc, 2), 300.0)}
        x = oc.column_features(d, st)
        coslat = np.sqrt(g.C[:, 0] ** 2 + g.C[:, 1] ** 2)
        eu = np.max(np.abs(x[:, 6] - U * coslat))
        ev = np.max(np.abs(x[:, 8]))
        errs.append(max(eu, ev))
    assert errs[-1] < 0.01 * U
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_features_of_the_reference_state_at_rest_vanish():
    d = _dycore(2, 6)
    g = d.g
    th, ex = d.reference_state()
    st = {"vn": np.zeros((g.ne, 6)), "w": np.zeros((g.nc, 7)), "exner": np.tile(ex, (g.nc, 1)),
          "theta_v": np.tile(th, (g.nc, 1))}
    x = oc.column_features(d, st)
    assert x.shape == (g.nc, 30) and np.all(x == 0.0)
    e = oc.edge_features(d, st, x)
    assert e.shape == (g.ne, 66) and np.all(e == 0.0)


def test_w_feature_is_the_full_level_mean_and_edge_features_take_both_sides():
    d = _dycore(1, 4)
    g = d.g
    rng = np.random.default_rng(3)
    st = {"vn": rng.standard_normal((g.ne, 4)), "w": rng.standard_normal((g.nc, 5)),
          "exner": np.ones((g.nc, 4)), "theta_v": np.full((g.nc, 4), 300.0)}
    x = oc.column_features(d, st)
    for c in (0, 7, g.nc - 1):
        for k in range(4):
            assert x[c, k] == 0.5 * (st["w"][c, k] + st["w"][c, k + 1])
    e = oc.edge_features(d, st, x)
    for ed in (0, 11, g.ne - 1):
        c0, c1 = g.e2c[ed]
        assert np.array_equal(e[ed, :20], x[c0]) and np.array_equal(e[ed, 20:40], x[c1])
        assert np.array_equal(e[ed, 40:], st["vn"][ed])


def test_targets_vanish_between_identical_steps():
    d = _dycore(1, 8, ndyn=3)
    grid = make_grid(1)
    st = jw_type_state(grid, make_vct(8), seed=1)
    st["exner_pr"] = d.initial_exner_pr(st["exner"])
    a, b = d.step(st), d.step(st)
    cy, ey = oc.targets(a, b)
    assert cy.shape == (d.g.nc, 23) and ey.shape == (d.g.ne, 8)
    assert np.all(cy == 0.0) and np.all(ey == 0.0)


def _zero_net(n_in, n_hid, n_out, b3):
    parts = [np.zeros(n_hid * n_in), np.zeros(n_hid), np.zeros(n_hid * n_hid), np.zeros(n_hid),
             np.zeros(n_out * n_hid), np.full(n_out, b3)]
    return np.concatenate(parts)


def test_constant_output_network_adds_closed_form_increments_and_keeps_rho():
    """With W = 0 the network outputs b3; the increment is b3 y_std + y_mean."""
    nlev, H = 4, 8
    d = _dycore(1, nlev)
    g = d.g
    rng = np.random.default_rng(5)
    st = {"vn": rng.standard_normal((g.ne, nlev)), "w": rng.standard_normal((g.nc, nlev + 1)),
          "rho": 1.0 + rng.random((g.nc, nlev)), "exner": 1.0 + 0.01 * rng.random((g.nc, nlev)),
          "theta_v": 300.0 + rng.random((g.nc, nlev)), "exner_pr": rng.random((g.nc, nlev))}
    ci, co, ei, eo = 5 * nlev, 3 * nlev - 1, 11 * nlev, nlev
    col = (_zero_net(ci, H, co, 0.5), (ci, H, co),
           (np.zeros(ci), np.ones(ci), np.full(co, 1e-3), np.full(co, 2.0)))
    edge = (_zero_net(ei, H, eo, -2.0), (ei, H, eo),
            (np.zeros(ei), np.ones(ei), np.zeros(eo), np.full(eo, 0.25)))
    cx = oc.column_features(d, st)
    inc_c, y_c = oc.network(*col, cx)
    inc_e, y_e = oc.network(*edge, oc.edge_features(d, st, cx))
    np.testing.assert_allclose(inc_c, 0.5 * 2.0 + 1e-3, rtol=0, atol=1e-15)
    np.testing.assert_allclose(inc_e, -0.5, rtol=0, atol=1e-15)
    out = oc.apply(st, inc_c, inc_e)
    assert np.array_equal(out["rho"], st["rho"]) and np.array_equal(out["exner_pr"], st["exner_pr"])
    assert np.array_equal(out["w"][:, [0, -1]], st["w"][:, [0, -1]])
    np.testing.assert_allclose(out["w"][:, 1:-1] - st["w"][:, 1:-1], 1.001, atol=1e-12)
    np.testing.assert_allclose(out["vn"] - st["vn"], -0.5, atol=1e-12)
    assert oc.check_value(y_c, y_e, out) == pytest.approx(2.0)


def test_check_value_is_nan_for_a_non_finite_rho():
    nlev = 3
    st = {"vn": np.zeros((6, nlev)), "w": np.zeros((4, nlev + 1)), "rho": np.ones((4, nlev)),
          "exner": np.ones((4, nlev)), "theta_v": np.ones((4, nlev))}
    st["rho"][2, 1] = np.nan
    assert np.isnan(oc.check_value(np.zeros((4, 8)), np.zeros((6, 3)), st))
    st["rho"][2, 1] = 1.0
    assert oc.check_value(np.full((4, 8), 3.0), np.full((6, 3), 1.0), st) == 3.0


def test_rejected_correction_returns_the_plain_step():
    nlev, H = 6, 8
    grid = make_grid(1)
    z = make_vct(nlev)
    red = Dycore(grid, z, DycoreParams(dtime=600.0, ndyn_substeps=4))
    pl = Dycore(grid, z, DycoreParams(dtime=600.0, ndyn_substeps=5))
    st = jw_type_state(grid, z, seed=2)
    st["exner_pr"] = pl.initial_exner_pr(st["exner"])
    ci, co, ei, eo = 5 * nlev, 3 * nlev - 1, 11 * nlev, nlev
    col = (_zero_net(ci, H, co, 1.0), (ci, H, co), (np.zeros(ci), np.ones(ci), np.zeros(co), np.ones(co)))
    edge = (_zero_net(ei, H, eo, 1.0), (ei, H, eo), (np.zeros(ei), np.ones(ei), np.zeros(eo), np.ones(eo)))
    out, fb, r = oc.step_learned(red, pl, col, edge, st, max_norm=0.5)
    ref = pl.step(st)
    assert fb and r == 1.0
    assert all(np.array_equal(out[k], ref[k]) for k in ref)
    out, fb, r = oc.step_learned(red, pl, col, edge, st, max_norm=1.0)
    sr = red.step(st)
    assert not fb and np.array_equal(out["rho"], sr["rho"])
    np.testing.assert_allclose(out["vn"] - sr["vn"], 1.0, atol=1e-9)


def test_gelu_network_matches_hand_evaluated_single_unit():
    """One hidden unit per layer: y = w3 GELU(w2 GELU(w1 x + b1) + b2) + b3."""
    p = np.array([2.0, 0.1, -1.5, 0.2, 3.0, -0.4])
    # raw input 0.55 with mean 0.2 and std 0.5 normalises to 0.7
    h1 = omlp.gelu(2.0 * 0.7 + 0.1)
    h2 = omlp.gelu(-1.5 * h1 + 0.2)
    inc, y = oc.network(p, (1, 1, 1), (np.array([0.2]), np.array([0.5]), np.array([1.0]), np.array([2.0])),
                        np.array([[0.55]]))
    assert y[0, 0] == pytest.approx(3.0 * h2 - 0.4, rel=1e-14)
    assert inc[0, 0] == pytest.approx((3.0 * h2 - 0.4) * 2.0 + 1.0, rel=1e-14)
