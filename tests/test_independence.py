"""The oracle and the product path stay apart (read from the sources, no GPU).

* Nothing in the package (Python binding, build script, CUDA and C++ sources)
  imports, includes or opens anything under ``oracle/``: the product path has
  no CPU fallback and no oracle arithmetic.
* The oracle imports nothing from the package.
* The shared input generators (``icon_inputs/``) import neither.
* Outside tests, only ``__graft_entry__.smoke`` and ``bench.py``'s CPU
  baseline and reference arm reach the oracle."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2608_21150_gb300")


def _imports(path):
    mods = set()
    for node in ast.walk(ast.parse(open(path).read())):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _py(d):
    return [f for f in glob.glob(os.path.join(d, "**", "*.py"), recursive=True) if "__pycache__" not in f]


def test_package_never_reaches_the_oracle():
    for f in _py(PKG):
        assert "oracle" not in _imports(f), f
        assert "icon_inputs" not in _imports(f), f
    for f in glob.glob(os.path.join(PKG, "csrc", "*")):
        src = open(f, errors="replace").read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), f
        assert "oracle/" not in src, f


def test_oracle_and_inputs_never_reach_the_package():
    for f in _py(os.path.join(ROOT, "oracle")):
        assert "paper_2608_21150_gb300" not in _imports(f), f
    for f in _py(os.path.join(ROOT, "icon_inputs")):
        assert not {"oracle", "paper_2608_21150_gb300"} & _imports(f), f


def test_only_smoke_and_the_cpu_baseline_reach_the_oracle_outside_tests():
    entry = ast.parse(open(os.path.join(ROOT, "__graft_entry__.py")).read())
    for fn in entry.body:
        if isinstance(fn, ast.FunctionDef):
            uses = any(isinstance(n, (ast.Import, ast.ImportFrom)) and "oracle" in ast.unparse(n) for n in ast.walk(fn))
            assert uses == (fn.name == "smoke"), fn.name
    bench = ast.parse(open(os.path.join(ROOT, "bench.py")).read())

    def reaches(fn):
        """Names, attributes and imports that mention the oracle, and source text
        that imports it (the child process of the CPU sample); other strings do
        not count."""
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and "oracle" in n.id:
                return True
            if isinstance(n, ast.Attribute) and "oracle" in n.attr:
                return True
            if isinstance(n, (ast.Import, ast.ImportFrom)) and "oracle" in ast.unparse(n):
                return True
            if isinstance(n, ast.Constant) and isinstance(n.value, str) and re.search(r"(import|from) oracle", n.value):
                return True
        return False

    reaching = {fn.name for fn in bench.body if isinstance(fn, ast.FunctionDef)
                and reaches(fn) and fn.name not in ("cpu_baseline", "run_reference")}
    # oracle_sample runs the oracle in a child process for those two
    assert reaching <= {"oracle_sample"}, reaching
    assert "oracle" not in {m for m in _imports(os.path.join(ROOT, "bench.py"))}
