"""The ctypes mirrors of the public structs in the Python binding have the
layout the C header gives them: a C program compiled against
include/icon_dycore.h prints each struct's size and every field's offset,
and they must equal ctypes' (a field added to the header but not to the
binding, or in another order, shifts every later field)."""
import os
import shutil
import subprocess

import pytest

from c_harness import ROOT


def test_binding_structs_match_the_header(built_lib, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    import ctypes
    from paper_2608_21150_gb300 import _binding as B
    structs = [B.icon_grid_desc_t, B.icon_dycore_params_t, B.icon_state_t]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "icon_dycore.h"', "int main(void) {"]
    for s in structs:
        n = s.__name__
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (n, n))
        for f, _ in s._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (n, f, n, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    c = dict(line.split() for line in out if line.strip())
    for s in structs:
        n = s.__name__
        assert int(c[n]) == ctypes.sizeof(s), n
        for f, _ in s._fields_:
            assert int(c[n + "." + f]) == getattr(s, f).offset, (n, f)
