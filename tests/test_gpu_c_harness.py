"""The C-ABI from plain C (tests/c/abi_harness.c): argument checks and two
steps of a host-memory state; the result equals, bit for bit, the same two
steps through the Python binding."""
import subprocess

import numpy as np
import pytest

from c_harness import FIELDS, build_harness, read_state, write_inputs
from parity import setup

pytestmark = pytest.mark.gpu


def test_c_harness_steps_like_the_binding(built_lib, cuda, tmp_path):
    import paper_2608_21150_gb300 as P
    grid, z, op, od, st = setup(2, 30, 1800.0)
    write_inputs(str(tmp_path), grid, z, st)
    exe = str(tmp_path / "abi_harness")
    build_harness(exe)
    r = subprocess.run([exe], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    got = read_state(str(tmp_path / "out.bin"), st)
    g = P.Grid(grid)
    d = P.Dycore(g, z, dict(dtime=1800.0, autotune=0, synchronous=1))
    host = {k: np.ascontiguousarray(st[k]).copy() for k in FIELDS}
    for _ in range(2):
        d.step(host)
    for k in FIELDS:
        assert np.array_equal(got[k], host[k]), k
