"""Helpers for the plain-C and Fortran uses of the C-ABI: the binary input
files both read (grid.bin, z_ifc.bin, state.bin) and the harness build."""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("vn", "w", "rho", "exner", "theta_v", "exner_pr")


def write_inputs(directory, grid, z, st):
    nlev = z.size - 1
    with open(os.path.join(directory, "grid.bin"), "wb") as f:
        np.array([grid.n_cells, grid.n_edges, grid.n_verts, nlev], dtype=np.int32).tofile(f)
        for a in (grid.c2v, grid.c2e, grid.e2c, grid.e2v, grid.v2e, grid.v2c):
            np.ascontiguousarray(a, dtype=np.int32).tofile(f)
        for a in (grid.cell_xyz, grid.vert_xyz, grid.edge_xyz):
            np.ascontiguousarray(a, dtype=np.float64).tofile(f)
    np.ascontiguousarray(z, dtype=np.float64).tofile(os.path.join(directory, "z_ifc.bin"))
    with open(os.path.join(directory, "state.bin"), "wb") as f:
        for k in FIELDS:
            np.ascontiguousarray(st[k], dtype=np.float64).tofile(f)


def read_state(path, like):
    raw = np.fromfile(path, dtype=np.float64)
    out, off = {}, 0
    for k in FIELDS:
        n = like[k].size
        out[k] = raw[off:off + n].reshape(like[k].shape)
        off += n
    assert off == raw.size
    return out


def build_harness(out_path):
    """Compile tests/c/abi_harness.c as C99 against include/ and the built library."""
    from paper_2608_21150_gb300.build import LIB
    libdir = os.path.dirname(LIB)
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_harness.c"), "-o", out_path, "-L", libdir, "-licondycore",
           "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
