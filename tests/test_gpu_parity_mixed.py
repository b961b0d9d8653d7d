"""Mixed precision (FP32 stencils, FP64 prognostic updates; the column solve
in double-word FP32, ICON_PREC_MIXED, or in FP64, ICON_PREC_MIXED_F64COL)
against the FP64 oracle.  Tolerances come from FP32 rounding (6e-8)
amplified by the cancellation of reference and perturbation parts in the
stencils."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    return P


MODES = ["dw", "f64col"]


def make(P, grid, z, op, mode="dw", **over):
    g = P.Grid(grid, radius=op.radius)
    prec = P.ICON_PREC_MIXED_F64COL if mode == "f64col" else P.ICON_PREC_MIXED
    return g, P.Dycore(g, z, gpu_params(op, precision=prec, **over))


@pytest.mark.parametrize("mode", MODES)
def test_mixed_step_close_to_fp64_oracle(lib, cuda, mode):
    grid, z, op, od, st = setup(2, 30, 1800.0, rayleigh=0.05)
    g, d = make(lib, grid, z, op, mode, rayleigh_coeff=0.05)
    t = to_torch(st, cuda)
    ref = dict(st)
    errs = []
    for n in range(1, 11):
        ref = od.step(ref)
        d.step(t)
        errs.append(rel_err(to_numpy(t), ref, od))
    print("mixed vs oracle, step 1:", errs[0])
    print("mixed vs oracle, step 10:", errs[-1])
    assert max(errs[0].values()) < 2e-5, errs[0]
    assert max(errs[-1].values()) < 1e-3, errs[-1]


@pytest.mark.parametrize("mode", MODES)
def test_mixed_conserves_mass_to_fp64_rounding(lib, cuda, mode):
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make(lib, grid, z, op, mode)
    t = to_torch(st, cuda)
    area = od.g.cell_area[:, None]

    def mass(s):
        return float(np.sum(area * s["rho"] * od.v.dz[None, :]))

    m0 = mass(st)
    for _ in range(10):
        d.step(t)
    assert abs(mass(to_numpy(t)) / m0 - 1) < 1e-13


@pytest.mark.parametrize("mode", MODES)
def test_mixed_resting_atmosphere_stays_at_rest(lib, cuda, mode):
    import torch
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make(lib, grid, z, op, mode)
    th, ex = d.reference_state()
    nc, ne, nlev = grid.n_cells, grid.n_edges, z.size - 1
    rest = dict(vn=np.zeros((ne, nlev)), w=np.zeros((nc, nlev + 1)), theta_v=np.tile(th, (nc, 1)),
                exner=np.tile(ex, (nc, 1)))
    rest["rho"] = op.p00 * rest["exner"] ** (op.cvd / op.rd) / (op.rd * rest["theta_v"])
    rest["exner_pr"] = np.zeros((nc, nlev))
    t = to_torch(rest, cuda)
    for _ in range(10):
        d.step(t)
    assert float(torch.max(torch.abs(t["vn"]))) <= 1e-12
    assert float(torch.max(torch.abs(t["w"]))) <= 1e-12


def test_mixed_stage_entry_is_fp64_only(lib, cuda):
    import torch
    grid, z, op, od, st = setup(1, 30, 1800.0)
    g, d = make(lib, grid, z, op)
    t = to_torch(st, cuda)
    with pytest.raises(lib.IconError) as e:
        d.velocity_tendencies(t["vn"], t["w"], torch.empty_like(t["vn"]), torch.empty_like(t["w"]))
    assert e.value.code == lib.ICON_ERR_UNSUPPORTED


def test_fp64_column_of_the_mixed_step_is_closer_to_fp64_than_the_double_word_one(lib, cuda):
    """The two mixed modes share every FP32 stencil; only the column solve's
    arithmetic differs, and its FP64 form follows the FP64 oracle at least as
    closely in w (the field the solve decides) after one step."""
    grid, z, op, od, st = setup(2, 30, 1800.0, rayleigh=0.05)
    ref = od.step(st)
    errs = {}
    for mode in MODES:
        g, d = make(lib, grid, z, op, mode, rayleigh_coeff=0.05)
        t = to_torch(st, cuda)
        d.step(t)
        errs[mode] = rel_err(to_numpy(t), ref, od)
    assert errs["f64col"]["w"] <= errs["dw"]["w"] * 1.5, errs
    assert all(e < 2e-5 for e in errs["f64col"].values()), errs
