"""Writes tests/golden/probtest_r2b2_l30.json: probtest ensemble spreads of the
FP64 oracle (oracle/probtest.py) for the R2B2 L30 experiment, at two
perturbation sizes: 1e-14 (double-precision rounding differences, for the
FP64 GPU run) and 1e-7 (about the FP32 unit roundoff, for the mixed-precision
run).  Calls only oracle/ and icon_inputs/.  Run from the repository root:
    python tests/golden/make_probtest.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from icon_inputs import make_grid, make_vct, jw_type_state  # noqa: E402
from oracle import Dycore, DycoreParams  # noqa: E402
from oracle import probtest  # noqa: E402

EXPERIMENT = dict(bisections=2, nlev=30, dtime=1800.0, ndyn_substeps=5, rayleigh_coeff=0.05, seed=0, nsteps=10)
MEMBERS = list(range(1, 11))
EPS = (1e-14, 1e-7)


def main():
    e = EXPERIMENT
    grid, z = make_grid(e["bisections"]), make_vct(e["nlev"])
    d = Dycore(grid, z, DycoreParams(dtime=e["dtime"], ndyn_substeps=e["ndyn_substeps"],
                                     rayleigh_coeff=e["rayleigh_coeff"]))
    st0 = jw_type_state(grid, z, seed=e["seed"])
    st0["exner_pr"] = d.initial_exner_pr(st0["exner"])
    control = probtest.control_run(d, st0, e["nsteps"])
    out = {"experiment": e, "members": MEMBERS, "perturbed": ["vn", "rho", "exner", "theta_v"],
           "norm": "per field max |x - control| / max |control| (exner, theta_v as deviations from the "
                   "reference profiles), max over members, per step",
           "spread": {}}
    for eps in EPS:
        out["spread"]["%g" % eps] = probtest.ensemble_spread(d, st0, eps, MEMBERS, e["nsteps"], control)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "probtest_r2b2_l30.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
