"""GPU (C-ABI, CUDA kernels) vs FP64 CPU oracle on identical seeded inputs.

Mirrors the paper's verification hierarchy (Sec. 4.4): stage-level
comparison of code segments by relative error with tolerance 1e-12, and
whole-run comparison.  Tolerances: 1e-12 relative after one step, 1e-9 after
ten steps (per field, inf-norm, exner/theta_v as deviations from the
reference profiles)."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(built_lib, cuda):
    import paper_2608_21150_gb300 as P
    return P


def make_gpu(P, grid, z, op, **over):
    g = P.Grid(grid, radius=op.radius)
    return g, P.Dycore(g, z, gpu_params(op, **over))


def test_velocity_tendencies_parity(lib, cuda):
    import torch
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make_gpu(lib, grid, z, op)
    # a nonzero w so that every term of the w tendency is exercised
    rng = np.random.default_rng(7)
    w = 0.05 * rng.standard_normal(st["w"].shape)
    w[:, 0] = 0.0
    w[:, -1] = 0.0
    ref_vn, ref_w, _ = od.velocity_tendencies(st["vn"], w)
    t = to_torch(dict(vn=st["vn"], w=w), cuda)
    ddt_vn = torch.empty_like(t["vn"])
    ddt_w = torch.empty_like(t["w"])
    d.velocity_tendencies(t["vn"], t["w"], ddt_vn, ddt_w)
    e_vn = np.max(np.abs(ddt_vn.cpu().numpy() - ref_vn)) / np.max(np.abs(ref_vn))
    e_w = np.max(np.abs(ddt_w.cpu().numpy() - ref_w)) / np.max(np.abs(ref_w))
    assert e_vn < 1e-12 and e_w < 1e-12, (e_vn, e_w)


def test_substep_parity(lib, cuda):
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make_gpu(lib, grid, z, op)
    ref = od.substep(dict(st))
    t = to_torch(st, cuda)
    d.nh_solve(t)
    err = rel_err(to_numpy(t), ref, od)
    assert max(err.values()) < 1e-12, err


def test_diffusion_parity(lib, cuda):
    grid, z, op, od, st = setup(2, 30, 1800.0)
    st = od.substep(st)  # a state with nonzero w
    g, d = make_gpu(lib, grid, z, op)
    ref = od.diffusion(dict(st))
    t = to_torch(st, cuda)
    d.nh_diff(t)
    err = rel_err(to_numpy(t), ref, od)
    assert max(err.values()) < 1e-12, err


@pytest.mark.parametrize("use_graph", [0, 1])
def test_step_parity_r2b2_1_and_10_steps(lib, cuda, use_graph):
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make_gpu(lib, grid, z, op, use_graph=use_graph)
    t = to_torch(st, cuda)
    ref = dict(st)
    for n in range(1, 11):
        ref = od.step(ref)
        d.step(t)
        if n == 1:
            err1 = rel_err(to_numpy(t), ref, od)
            assert max(err1.values()) < 1e-12, err1
    err10 = rel_err(to_numpy(t), ref, od)
    assert max(err10.values()) < 1e-9, err10


def test_resting_atmosphere_gpu(lib, cuda):
    import torch
    grid, z, op, od, st = setup(2, 30, 1800.0)
    g, d = make_gpu(lib, grid, z, op)
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
