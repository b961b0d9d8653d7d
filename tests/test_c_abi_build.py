"""The public header is plain C: a C99 program using it compiles with
warnings as errors and links against the library (no GPU needed); the
Fortran interface module compiles where a Fortran compiler exists."""
import os
import shutil
import subprocess

import pytest

from c_harness import ROOT, build_harness


def test_c_harness_compiles_and_links(built_lib, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "abi_harness")
    build_harness(exe)
    assert os.path.exists(exe)


def test_fortran_interface_module_compiles(tmp_path):
    fc = shutil.which("gfortran")
    if fc is None:
        pytest.skip("no Fortran compiler on this machine")
    for f in ("icon_dycore.f90", "example_step.f90"):
        subprocess.run([fc, "-std=f2008", "-fsyntax-only", "-J", str(tmp_path), os.path.join(ROOT, "fortran", f)],
                       check=True, cwd=tmp_path)
