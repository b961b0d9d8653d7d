"""The mixed mode's column solve computes in double-word FP32 arithmetic (an
unevaluated sum of two floats, about 48 significant bits) instead of FP64.
On identical inputs -- those of a real substep's corrector solve -- it must
agree with the FP64 solve to well below the mixed mode's FP32 stencil error."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("corrector", [False, True])
def test_double_word_column_solve_matches_fp64(built_lib, cuda, corrector):
    import torch
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(3, 90, 900.0, rayleigh=0.05, seed=5)
    params = gpu_params(op, rayleigh_coeff=0.05)
    g = P.Grid(grid, radius=op.radius)
    d = P.Dycore(g, z, params)
    nc, nlev = grid.n_cells, z.size - 1
    t = to_torch(st, cuda)
    for _ in range(2):                      # a developed state
        d.nh_solve(t)
    now = {k: v.clone() for k, v in t.items()}
    d.nh_solve(t)
    f = {}
    for name, n in (("rho_p", nc * nlev), ("theta_p", nc * nlev), ("ddt_w0", nc * (nlev + 1)),
                    ("ddt_w1", nc * (nlev + 1)), ("div_m", nc * nlev), ("div_t", nc * nlev)):
        f[name] = torch.empty(n, dtype=torch.float64, device=cuda)
        d.debug_field(name, f[name])
    extra = dict(rho_pred=f["rho_p"], theta_pred=f["theta_p"], ddt_w1=f["ddt_w1"]) if corrector else {}
    outs = {}
    for prec in (P.ICON_PREC_FP64, P.ICON_PREC_MIXED):
        pp = dict(params, precision=prec, synchronous=1)
        out = {k: torch.empty_like(now[k]) for k in ("w", "rho", "exner", "theta_v")}
        P.column_solve_noalloc(z, pp, now["w"], now["rho"], now["exner"], now["theta_v"], f["ddt_w0"],
                               f["div_m"], f["div_t"], out["w"], out["rho"], out["exner"], out["theta_v"], **extra)
        outs[prec] = to_numpy(out)
    th_ref, ex_ref = od.reference_state()
    errs = {}
    for k in ("w", "rho", "exner", "theta_v"):
        a, b = outs[P.ICON_PREC_MIXED][k], outs[P.ICON_PREC_FP64][k]
        if k == "exner":
            a, b = a - ex_ref, b - ex_ref
        if k == "theta_v":
            a, b = a - th_ref, b - th_ref
        if k == "rho":   # relative to the step's change of rho, the quantity the solve computes
            b0 = now["rho"].cpu().numpy()
            a, b = a - b0, b - b0
        errs[k] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert all(e < 1e-9 for e in errs.values()), errs
    print(errs)
