"""The C-ABI from Fortran through iso_c_binding (Sec. 4.3: the dycore called
by a Fortran host model): fortran/icon_dycore.f90 and fortran/example_step.f90
compiled with gfortran and linked against the library, two steps of a
host-memory R2B2 L30 state.  The result equals, bit for bit, the same two
steps through the Python binding, and the oracle's two steps to 1e-11.
Skipped where no Fortran compiler is installed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from c_harness import FIELDS, ROOT, read_state, write_inputs
from parity import setup, rel_err

pytestmark = pytest.mark.gpu


def test_fortran_example_steps_like_the_binding_and_the_oracle(built_lib, cuda, tmp_path):
    fc = shutil.which("gfortran")
    if fc is None:
        pytest.skip("no Fortran compiler on this machine")
    import paper_2608_21150_gb300 as P
    from paper_2608_21150_gb300.build import LIB
    libdir = os.path.dirname(LIB)
    grid, z, op, od, st = setup(2, 30, 1800.0)
    write_inputs(str(tmp_path), grid, z, st)
    exe = str(tmp_path / "example_step")
    subprocess.run([fc, "-std=f2008", "-O2", "-J", str(tmp_path), os.path.join(ROOT, "fortran", "icon_dycore.f90"),
                    os.path.join(ROOT, "fortran", "example_step.f90"), "-o", exe, "-L", libdir, "-licondycore",
                    "-Wl,-rpath," + libdir], check=True, cwd=tmp_path)
    r = subprocess.run([exe], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    got = read_state(str(tmp_path / "out.bin"), st)
    d = P.Dycore(P.Grid(grid), z, dict(dtime=1800.0, autotune=0, synchronous=1))
    host = {k: np.ascontiguousarray(st[k]).copy() for k in FIELDS}
    for _ in range(2):
        d.step(host)
    for k in FIELDS:
        assert np.array_equal(got[k], host[k]), k
    ref = od.step(od.step(st))
    errs = rel_err(got, ref, od)
    assert max(errs.values()) < 1e-11, errs
