"""The probtest ensemble machinery (oracle/probtest.py, icon_inputs.perturb)
and its stored tolerances (tests/golden/probtest_r2b2_l30.json, written by
tests/golden/make_probtest.py from the oracle only)."""
import json
import os

import numpy as np

from icon_inputs import make_grid, make_vct, jw_type_state, perturb_state
from oracle import Dycore, DycoreParams
from oracle import probtest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "probtest_r2b2_l30.json")


def test_perturbation_is_seeded_relative_and_bounded():
    g, z = make_grid(1), make_vct(8)
    st = jw_type_state(g, z, seed=0)
    a, b, c = perturb_state(st, 1e-3, 5), perturb_state(st, 1e-3, 5), perturb_state(st, 1e-3, 6)
    for k in ("vn", "rho", "exner", "theta_v"):
        assert np.array_equal(a[k], b[k]) and not np.array_equal(a[k], c[k])
        r = np.abs(a[k] - st[k]) / np.maximum(np.abs(st[k]), 1e-300)
        assert np.all(r <= 1e-3 * (1 + 1e-12))
    assert np.array_equal(a["w"], st["w"])


def test_zero_perturbation_gives_zero_spread_and_nonzero_eps_a_positive_one():
    g, z = make_grid(1), make_vct(10)
    d = Dycore(g, z, DycoreParams(dtime=3600.0))
    st = jw_type_state(g, z, seed=1)
    st["exner_pr"] = d.initial_exner_pr(st["exner"])
    ctl = probtest.control_run(d, st, 2)
    s0 = probtest.ensemble_spread(d, st, 0.0, [1, 2], 2, ctl)
    assert all(v == 0.0 for sp in s0.values() for v in sp)
    s1 = probtest.ensemble_spread(d, st, 1e-10, [1, 2], 2, ctl)
    assert all(np.isfinite(v) and v > 0.0 for sp in s1.values() for v in sp)


def test_golden_spreads_grow_linearly_with_the_perturbation():
    """Over 10 steps the ensemble stays in the linear regime: spreads at
    eps = 1e-7 are 1e7 times those at 1e-14 within a factor of 10."""
    j = json.load(open(GOLDEN))
    lo, hi = j["spread"]["1e-14"], j["spread"]["1e-07"]
    assert set(lo) == set(probtest.FIELDS) and len(lo["vn"]) == j["experiment"]["nsteps"]
    for k in lo:
        for a, b in zip(lo[k], hi[k]):
            assert a > 0 and 1e6 < b / a < 1e8, (k, a, b)
