"""Probtest verification of the GPU runs (the paper's third level, Sec. 4.4):
the FP64 and mixed-precision GPU runs of the R2B2 L30 experiment, compared
with the oracle's unperturbed run at each of 10 steps (50 substeps), must stay
within FACTOR times the spread of the oracle's perturbed ensemble
(tests/golden/probtest_r2b2_l30.json): perturbations of 1e-14 for FP64 (the
size of double-precision rounding differences) and 1e-7 for mixed precision
(about the FP32 unit roundoff)."""
import json
import os

import pytest

from icon_inputs import make_grid, make_vct, jw_type_state
from oracle import Dycore as OracleDycore, DycoreParams
from oracle import probtest
from parity import gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "probtest_r2b2_l30.json")
FACTOR = 5.0


@pytest.fixture(scope="module")
def reference():
    j = json.load(open(GOLDEN))
    e = j["experiment"]
    grid, z = make_grid(e["bisections"]), make_vct(e["nlev"])
    op = DycoreParams(dtime=e["dtime"], ndyn_substeps=e["ndyn_substeps"], rayleigh_coeff=e["rayleigh_coeff"])
    od = OracleDycore(grid, z, op)
    st0 = jw_type_state(grid, z, seed=e["seed"])
    st0["exner_pr"] = od.initial_exner_pr(st0["exner"])
    control = probtest.control_run(od, st0, e["nsteps"])
    return dict(j=j, grid=grid, z=z, op=op, od=od, st0=st0, control=control)


@pytest.mark.parametrize("mode,eps", [("fp64", "1e-14"), ("mixed", "1e-07")])
def test_gpu_run_within_probtest_tolerances(built_lib, cuda, reference, mode, eps):
    import paper_2608_21150_gb300 as P
    r = reference
    prec = P.ICON_PREC_MIXED if mode == "mixed" else P.ICON_PREC_FP64
    g = P.Grid(r["grid"], radius=r["op"].radius)
    d = P.Dycore(g, r["z"], gpu_params(r["op"], precision=prec))
    t = to_torch(r["st0"], cuda)
    spread = r["j"]["spread"][eps]
    worst = {}
    for n, ctl in enumerate(r["control"]):
        d.step(t)
        diff = probtest.differences(to_numpy(t), ctl, r["od"])
        for k, v in diff.items():
            ratio = v / (FACTOR * spread[k][n])
            worst[k] = max(worst.get(k, 0.0), ratio)
            assert v <= FACTOR * spread[k][n], (mode, n + 1, k, v, spread[k][n])
    print(mode, "largest difference / tolerance per field over 10 steps:", worst)
    d.close()
    g.close()
