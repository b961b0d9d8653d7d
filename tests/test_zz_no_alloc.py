"""The allocation-free column solve (icon_column_solve_noalloc), for callers
that cannot allocate device memory when they call, against the column solve
inside icon_nh_solve.

icon_nh_solve runs a full substep; its last kernel is the corrector's column
solve.  The inputs of that solve are read back with icon_dycore_debug_field
(predicted rho/theta_v, both w tendencies, both flux divergences) and handed
to the allocation-free entry point together with the state at the start of
the substep; its outputs must equal the substep's w, rho, exner and theta_v
within the parity tolerance.  Two substeps in a row check that the static
scratch, which keeps the previous call's contents, needs no clearing.  This
file is collected last, so a run that stops at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from parity import setup, gpu_params, to_torch, to_numpy

pytestmark = pytest.mark.gpu


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


def test_noalloc_rejects_sizes_beyond_the_static_scratch(built_lib, cuda):
    """The limit is checked before any memory is touched or any kernel starts."""
    import ctypes
    import torch
    import paper_2608_21150_gb300 as P
    nlev = 90
    n_cols = 1_047_552 // (nlev + 1) + 1
    z = np.ascontiguousarray(np.linspace(30000.0, 0.0, nlev + 1))
    x = torch.zeros(8, dtype=torch.float64, device=cuda)
    p = P.default_params()
    rc = P.icon_column_solve_noalloc(n_cols, nlev, z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(p), *([x.data_ptr()] * 4), None, None, x.data_ptr(), None,
                                     *([x.data_ptr()] * 6))
    assert rc == P.ICON_ERR_ARG and b"static scratch" in P.icon_last_error()
