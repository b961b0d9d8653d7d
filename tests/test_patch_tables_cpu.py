"""The fused velocity-advection kernel's patch tables, built on the host by
csrc/patch_setup.cpp, checked without a GPU: tests/c/patch_tables_check.cpp
compiles against the library's host sources and verifies every local index
of every patch against the global connectivity, the own-cells-first order and
that each edge is written by exactly one patch, on grids from R2B0 (one patch
larger than the grid) to R2B4, for the library's patch size and for sizes
that leave ragged last patches."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from c_harness import ROOT
from icon_inputs import make_grid

CSRC = os.path.join(ROOT, "paper_2608_21150_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no g++ or CUDA headers")
    exe = str(tmp_path_factory.mktemp("patch") / "patch_tables_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", cuda_inc, "-I", CSRC,
                    os.path.join(ROOT, "tests", "c", "patch_tables_check.cpp"),
                    os.path.join(CSRC, "patch_setup.cpp"), os.path.join(CSRC, "grid_setup.cpp"), "-o", exe],
                   check=True)
    return exe


def write_grid(g, path):
    with open(path, "wb") as f:
        np.array([g.n_cells, g.n_edges, g.n_verts], np.int32).tofile(f)
        for name in ("c2v", "c2e", "e2c", "e2v", "v2e", "v2c"):
            np.ascontiguousarray(getattr(g, name), np.int32).tofile(f)
        for name in ("cell_xyz", "vert_xyz", "edge_xyz"):
            np.ascontiguousarray(getattr(g, name), np.float64).tofile(f)


@pytest.mark.parametrize("bisections", [0, 1, 2, 4])
@pytest.mark.parametrize("patch", [128, 100, 37])
def test_patch_tables_consistent(checker, tmp_path, bisections, patch):
    g = make_grid(bisections)
    path = str(tmp_path / "grid.bin")
    write_grid(g, path)
    out = subprocess.run([checker, path, str(patch)], capture_output=True, text=True, check=True).stdout.split()
    assert out[0] == "ok", out
    n_patches, max_e0, max_e1, max_c3, max_c0, max_v3, max_e4 = map(int, out[1:])
    assert n_patches == -(-g.n_cells // patch)
    own = min(patch, g.n_cells)
    # the own cells' edges, their cells, the halo cells and edges are all there
    assert 3 * own // 2 <= max_e4 <= 3 * own
    assert own <= max_c3 <= max_c0 <= g.n_cells
    assert max_e4 <= max_e1 <= max_e0 <= g.n_edges and max_v3 <= g.n_verts


def test_patch_tables_bad_size_refused(checker, tmp_path):
    path = str(tmp_path / "grid.bin")
    write_grid(make_grid(0), path)
    p = subprocess.run([checker, path, "0"], capture_output=True, text=True)
    assert p.returncode != 0 and "patch size must be positive" in p.stdout
