"""The allocation-free column solve (icon_column_solve_noalloc).

Some callers cannot allocate device memory when they call: a host model that
reserved nearly all device memory for its own arrays at start-up has no room
left for a dycore's work arrays.  This entry point runs the vertically
implicit column solve on the caller's arrays, with its scratch in a static
device array of the library, and allocates nothing.

Checked here, each time on two calls in a row (the static scratch keeps the
previous call's contents, so a second call shows that nothing needs
clearing):
* against the column solve inside icon_nh_solve (the substep's corrector
  solve, its inputs read back with icon_dycore_debug_field);
* against the oracle's column solve, predictor and corrector forms, FP64 and
  the mixed mode's double-word arithmetic;
* the size limit on both sides of the boundary (11 508 columns of 90 levels
  accepted, 11 509 refused) and an unknown precision refused.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu

LIMIT = 1_047_232          # column-levels of the static scratch


def _dev(a, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(cuda)


def test_noalloc_column_solve_matches_nh_solve(built_lib, cuda):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0, rayleigh=0.05)
    params = gpu_params(op, rayleigh_coeff=0.05)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, params)
    nc, nlev = grid.n_cells, z.size - 1
    t = to_torch(st, cuda)
    for call in range(2):
        now = {k: v.clone() for k, v in t.items()}
        d.nh_solve(t)
        fields = {}
        for name, n in (("rho_p", nc * nlev), ("theta_p", nc * nlev), ("ddt_w0", nc * (nlev + 1)),
                        ("ddt_w1", nc * (nlev + 1)), ("div_m", nc * nlev), ("div_t", nc * nlev)):
            fields[name] = torch.empty(n, dtype=torch.float64, device=cuda)
            d.debug_field(name, fields[name])
        out = {k: torch.empty_like(now[k]) for k in ("w", "rho", "exner", "theta_v")}
        P.column_solve_noalloc(z, params, now["w"], now["rho"], now["exner"], now["theta_v"],
                               fields["ddt_w0"], fields["div_m"], fields["div_t"], out["w"], out["rho"],
                               out["exner"], out["theta_v"], rho_pred=fields["rho_p"],
                               theta_pred=fields["theta_p"], ddt_w1=fields["ddt_w1"])
        ref = to_numpy({k: t[k] for k in out})
        got = to_numpy(out)
        th_ref, ex_ref = od.reference_state()
        for k in out:
            a, b = got[k], ref[k]
            if k == "exner":
                a, b = a - ex_ref, b - ex_ref
            if k == "theta_v":
                a, b = a - th_ref, b - th_ref
            err = np.max(np.abs(a - b)) / np.max(np.abs(b))
            assert err < 1e-12, (call, k, err)
    d.close()
    g.close()


def _oracle_solve_inputs(od, st):
    """Inputs of a substep's predictor and corrector column solves, computed
    with the oracle's own pieces (velocity tendencies, upwind edge values,
    flux divergences), and the oracle's solves on them."""
    p, v = od.p, od.v
    dt = p.dtime / p.ndyn_substeps
    vn, w, rho, theta = st["vn"], st["w"], st["rho"], st["theta_v"]
    ddt_vn0, ddt_w0, vt = od.velocity_tendencies(vn, w)
    pr = st["exner"] - v.exner_ref[None, :]
    pr_ex = od.extrapolate_exner(pr, st["exner_pr"])
    rho_e = od.upwind_edge_values(rho, vn, vt, dt)
    theta_e = od.upwind_edge_values(theta, vn, vt, dt)
    vn_pred = vn + dt * (ddt_vn0 - p.cpd * theta_e * od.grad_n(pr_ex))
    vf = od.flux_velocity(vn_pred)
    div_m, div_t = od.div(rho_e * vf), od.div(rho_e * theta_e * vf)
    th_ref = v.theta_ref[None, :]
    pred = od.vertical_solve(st, v.interp_ic(rho), v.interp_ic(theta), v.interp_ic(theta - th_ref),
                             div_m, div_t, ddt_w0, dt)
    ddt_w1 = od.velocity_tendencies(vn_pred, pred["w"])[1]
    ra = p.wgt_nnow_rth * rho + p.wgt_nnew_rth * pred["rho"]
    ta = p.wgt_nnow_rth * theta + p.wgt_nnew_rth * pred["theta_v"]
    corr = od.vertical_solve(st, v.interp_ic(ra), v.interp_ic(ta), v.interp_ic(ta - th_ref), div_m, div_t,
                             p.wgt_nnow_vel * ddt_w0 + p.wgt_nnew_vel * ddt_w1, dt)
    return dict(ddt_w0=ddt_w0, ddt_w1=ddt_w1, div_m=div_m, div_t=div_t, rho_p=pred["rho"],
                theta_p=pred["theta_v"]), pred, corr


@pytest.mark.parametrize("corrector", [False, True], ids=["predictor", "corrector"])
@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_noalloc_forms_match_the_oracle_solve(built_lib, cuda, corrector, mixed):
    """Both forms and both arithmetics against the oracle's column solve on the
    same inputs (a developed R2B2 L30 state, Rayleigh damping on).  FP64: the
    parity norm at 1e-12.  Mixed (double-word FP32, about 48 bits): 1e-9, with
    rho measured against its change over the solve."""
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0, rayleigh=0.05, seed=3)
    st = od.step(st)
    inp, pred, corr = _oracle_solve_inputs(od, st)
    ref = corr if corrector else pred
    params = gpu_params(op, rayleigh_coeff=0.05, precision=P.ICON_PREC_MIXED if mixed else P.ICON_PREC_FP64)
    now = to_torch({k: st[k] for k in ("w", "rho", "exner", "theta_v")}, cuda)
    f = {k: _dev(x, cuda) for k, x in inp.items()}
    extra = dict(rho_pred=f["rho_p"], theta_pred=f["theta_p"], ddt_w1=f["ddt_w1"]) if corrector else {}
    th_ref, ex_ref = od.reference_state()
    tol = 1e-9 if mixed else 1e-12
    first = None
    for call in range(2):
        out = {k: torch.full_like(now[k], np.nan) for k in now}
        P.column_solve_noalloc(z, params, now["w"], now["rho"], now["exner"], now["theta_v"], f["ddt_w0"],
                               f["div_m"], f["div_t"], out["w"], out["rho"], out["exner"], out["theta_v"], **extra)
        got = to_numpy(out)
        for k in ("w", "rho", "exner", "theta_v"):
            a, b = got[k], ref[k]
            if k == "exner":
                a, b = a - ex_ref, b - ex_ref
            if k == "theta_v":
                a, b = a - th_ref, b - th_ref
            if k == "rho" and mixed:
                a, b = a - st["rho"], b - st["rho"]
            err = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            assert err < tol, (call, k, err)
        if first is None:
            first = got
        else:
            for k in got:
                assert np.array_equal(got[k], first[k]), k


def test_noalloc_size_limit_boundary(built_lib, cuda):
    """At 90 levels, 11 508 columns (1 047 228 column-levels) fit the static
    scratch and are solved; 11 509 are refused before any GPU work.  The state
    is the resting reference atmosphere, which the solve keeps at rest."""
    import ctypes
    import torch
    import paper_2608_21150_gb300 as P
    from oracle import Dycore as OracleDycore, DycoreParams
    from icon_inputs import make_grid, make_vct
    nlev = 90
    n_ok = LIMIT // (nlev + 1)
    assert n_ok == 11508 and n_ok * (nlev + 1) <= LIMIT < (n_ok + 1) * (nlev + 1)
    z = make_vct(nlev)
    od = OracleDycore(make_grid(0), z, DycoreParams(dtime=360.0, rayleigh_coeff=0.05))
    th, ex = od.reference_state()
    p = od.p
    rho = p.p00 * ex ** (p.cvd / p.rd) / (p.rd * th)
    col = lambda x: torch.from_numpy(np.ascontiguousarray(np.tile(x, (n_ok, 1)))).to(cuda)  # noqa: E731
    w = torch.zeros((n_ok, nlev + 1), dtype=torch.float64, device=cuda)
    r, e, t = col(rho), col(ex), col(th)
    zero_c = torch.zeros((n_ok, nlev), dtype=torch.float64, device=cuda)
    params = dict(dtime=360.0, ndyn_substeps=5, rayleigh_coeff=0.05)
    for call in range(2):
        out = {k: torch.full_like(x, np.nan) for k, x in (("w", w), ("rho", r), ("exner", e), ("theta_v", t))}
        P.column_solve_noalloc(z, params, w, r, e, t, w, zero_c, zero_c, out["w"], out["rho"], out["exner"],
                               out["theta_v"])
        for k, x in out.items():
            assert bool(torch.isfinite(x).all()), (call, k)
        assert float(out["w"].abs().max()) < 1e-9
        assert float(((out["rho"] - r) / r).abs().max()) < 1e-12
    # one column more: refused with the limit in the message, the outputs untouched
    n_bad = n_ok + 1
    x = torch.zeros(8, dtype=torch.float64, device=cuda)
    pp = P.default_params()
    zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = P.icon_column_solve_noalloc(n_bad, nlev, zp, ctypes.byref(pp), *([x.data_ptr()] * 4), None, None,
                                     x.data_ptr(), None, *([x.data_ptr()] * 6))
    assert rc == P.ICON_ERR_ARG and b"static scratch" in P.icon_last_error()
    assert b"1047232" in P.icon_last_error()
    assert float(x.abs().max()) == 0.0
    # an unknown precision mode is refused (not run as FP64)
    pp.precision = 7
    rc = P.icon_column_solve_noalloc(2, nlev, zp, ctypes.byref(pp), *([x.data_ptr()] * 4), None, None,
                                     x.data_ptr(), None, *([x.data_ptr()] * 6))
    assert rc == P.ICON_ERR_ARG and b"precision" in P.icon_last_error()
