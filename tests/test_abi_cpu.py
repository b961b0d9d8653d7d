"""The C-ABI library builds, loads and exports every symbol the public header
declares; argument and grid validation run on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from icon_inputs import make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "icon_dycore.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(icon_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("icon_grid_create", "icon_grid_destroy", "icon_dycore_create", "icon_dycore_step",
              "icon_dycore_destroy", "icon_nh_solve", "icon_nh_diff", "icon_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (icon_\w+)", out))
    assert set(declared_functions()) <= exported


def test_params_defaults(built_lib):
    import paper_2608_21150_gb300 as P
    p = P.default_params()
    assert p.dtime == 1800.0 and p.ndyn_substeps == 5 and p.vwind_impl_wgt == 0.65
    assert p.precision == P.ICON_PREC_FP64 and p.use_graph == 1 and p.synchronous == 1
    assert abs(p.hdiff_k4 - 1 / 288) < 1e-18 and p.rayleigh_coeff == 0.0
    with pytest.raises(KeyError):
        P.default_params(no_such_field=1)


def _grid_err(P, grid, **kw):
    try:
        P.Grid(grid, **kw)
    except P.IconError as e:
        return e.code, str(e)
    return 0, ""


@pytest.mark.parametrize("corrupt", ["e2c_same", "c2e_range", "e2v_not_in_cell", "v2c_wrong", "coord"])
def test_grid_validation_rejects_inconsistent_tables(built_lib, corrupt):
    import paper_2608_21150_gb300 as P
    g = make_grid(1)
    if corrupt == "e2c_same":
        g.e2c[7, 1] = g.e2c[7, 0]
    elif corrupt == "c2e_range":
        g.c2e[3, 2] = g.n_edges
    elif corrupt == "e2v_not_in_cell":
        other = [v for v in range(g.n_verts) if v not in g.c2v[g.e2c[11]].ravel()][0]
        g.e2v[11, 0] = other
    elif corrupt == "v2c_wrong":
        g.v2c[20, 0] = (g.v2c[20, 0] + 37) % g.n_cells
    elif corrupt == "coord":
        g.cell_xyz[5] *= 1.5
    code, msg = _grid_err(P, g)
    assert code == P.ICON_ERR_GRID, msg


def test_valid_grid_passes_host_validation(built_lib):
    import paper_2608_21150_gb300 as P
    import torch
    if torch.cuda.is_available():
        pytest.skip("on a GPU machine the grid is created for real (GPU tests)")
    for base in (0, 1):
        code, msg = _grid_err(P, make_grid(1), index_base=base)
        # passes validation and only fails when it needs the (absent) device
        assert code == P.ICON_ERR_CUDA, msg


def test_null_arguments(built_lib):
    import paper_2608_21150_gb300 as P
    out = ctypes.c_void_p()
    assert P.icon_grid_create(None, ctypes.byref(out)) == P.ICON_ERR_ARG
    assert b"NULL" in P.icon_last_error()
    assert P.icon_grid_destroy(None) == P.ICON_OK
    assert P.icon_dycore_destroy(None) == P.ICON_OK
    assert P.icon_dycore_step(None, None) == P.ICON_ERR_ARG
    assert P.icon_dycore_synchronize(None) == P.ICON_ERR_ARG


def test_grid_validation_refuses_random_single_corruptions(built_lib):
    """Seeded sweep: one entry of one connectivity table set to another value
    (an in-range index, the pad value, or an out-of-range index), or one
    coordinate moved off the unit sphere.  Every such grid is refused on the
    host (ICON_ERR_GRID or ICON_ERR_ARG): none passes validation, which on this
    machine would surface as ICON_ERR_CUDA when the device is needed.  (A
    vertex row listing one of its edges or cells twice, dropping another, once
    passed: rows are now checked for repeats and against the vertex degree.)"""
    import paper_2608_21150_gb300 as P
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only sweep")
    rng = np.random.default_rng(2024)
    base = make_grid(1)
    counts = {"c2v": base.n_verts, "c2e": base.n_edges, "e2c": base.n_cells, "e2v": base.n_verts,
              "v2e": base.n_edges, "v2c": base.n_cells}
    refused = 0
    for trial in range(600):
        g = make_grid(1)
        if trial % 8 == 7:
            arr = (g.cell_xyz, g.vert_xyz, g.edge_xyz)[trial % 3]
            arr[rng.integers(arr.shape[0])] *= 1.0 + rng.uniform(0.01, 0.5)
        else:
            name = list(counts)[trial % 6]
            tab = getattr(g, name)
            i, j = rng.integers(tab.shape[0]), rng.integers(tab.shape[1])
            old = int(tab[i, j])
            kind = rng.integers(3)
            if kind == 0:
                new = int(rng.integers(counts[name]))
                if new == old:
                    new = (new + 1) % counts[name]
            elif kind == 1:
                new = -1 if old != -1 else 0
            else:
                new = counts[name] + int(rng.integers(1, 1000))
            tab[i, j] = new
        code, msg = _grid_err(P, g)
        assert code in (P.ICON_ERR_GRID, P.ICON_ERR_ARG), (trial, code, msg)
        refused += 1
    assert refused == 600
