"""Mutation check of the oracle's CPU pins (test infrastructure; not collected
by pytest).

Plants one mistake at a time in a copy of `oracle/` and runs the oracle's CPU
pin suites against it; a mutant that no pin fails "survives".  The mistakes
are the plausible slips of hand-written numerics:

  swap   a + b <-> a - b
  dropr  a + b -> a, a - b -> a     (a dropped term)
  neg    -x -> x                    (a lost sign)

at every such site of the chosen files, one site per mutant, identified by its
position in the syntax-tree walk.  Each mutant runs in its own directory under
_build/oracle_mutants/ (git-ignored) with `pytest -x`, several in parallel.

    python tests/oracle_mutation_sweep.py [--files oracle/dycore.py,...]
        [--jobs 8] [--out _build/oracle_mutants.jsonl] [--rerun previous.jsonl]
        [--suites tests/test_a.py,tests/test_b.py]

Writes one JSON line per mutant (file, kind, line, function, killed, first
failing test) and prints the survivors.  --rerun takes only the survivors of an
earlier output.  A full run over oracle/*.py (about 400 mutants) takes about
half an hour on 8 cores.
"""
import argparse
import ast
import copy
import json
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_SUITES = ["tests/test_probtest_cpu.py", "tests/test_oracle_closed_forms.py", "tests/test_oracle_terrain.py",
              "tests/test_oracle_corrector.py", "tests/test_oracle_pins.py"]
ORACLE_FILES = ["oracle/dycore.py", "oracle/vertical.py", "oracle/geometry.py", "oracle/diagnostics.py",
                "oracle/corrector.py", "oracle/mlp.py", "oracle/probtest.py", "oracle/terrain.py"]


def _is_site(node):
    if isinstance(node, ast.BinOp):
        return isinstance(node.op, (ast.Add, ast.Sub))
    if isinstance(node, ast.UnaryOp):
        return isinstance(node.op, ast.USub) and not isinstance(node.operand, ast.Constant)
    return False


class Sites(ast.NodeVisitor):
    """Mutation sites in walk order: (kind, line, col, function, index)."""

    def __init__(self):
        self.sites, self.stack, self.n = [], [], 0

    def visit_FunctionDef(self, node):
        self.stack.append(node.name)
        self.generic_visit(node)
        self.stack.pop()

    def generic_visit(self, node):
        if _is_site(node):
            f = ".".join(self.stack)
            kinds = ("swap", "dropr") if isinstance(node, ast.BinOp) else ("neg",)
            self.sites += [(k, node.lineno, node.col_offset, f, self.n) for k in kinds]
            self.n += 1
        super().generic_visit(node)


class Mutate(ast.NodeTransformer):
    """Applies one mutation at the site with the given walk-order index."""

    def __init__(self, kind, index):
        self.kind, self.index, self.n, self.done = kind, index, 0, False

    def generic_visit(self, node):
        if _is_site(node):
            mine = self.n == self.index
            self.n += 1
            if mine:
                self.done = True
                if self.kind == "swap":
                    node.op = ast.Sub() if isinstance(node.op, ast.Add) else ast.Add()
                elif self.kind == "dropr":
                    return self.visit(node.left)
                elif self.kind == "neg":
                    return self.visit(node.operand)
        return super().generic_visit(node)


def _run_one(mid, rel, tree, site, workdir, suites):
    d = os.path.join(workdir, str(mid))
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(d)
    for sub in ("oracle", "icon_inputs", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "*.o"))
    m = Mutate(site[0], site[4])
    mutated = m.visit(copy.deepcopy(tree))
    assert m.done, site
    with open(os.path.join(d, rel), "w") as f:
        f.write(ast.unparse(ast.fix_missing_locations(mutated)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    res = {"file": rel, "kind": site[0], "line": site[1], "col": site[2], "func": site[3], "index": site[4]}
    try:
        p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *suites],
                           cwd=d, env=env, capture_output=True, text=True, timeout=600)
        lines = p.stdout.strip().splitlines()
        res["killed"] = p.returncode != 0
        res["by"] = next((ln for ln in lines if ln.startswith(("FAILED", "ERROR"))), "")[:160]
    except subprocess.TimeoutExpired:
        res["killed"], res["by"] = True, "timeout"
    shutil.rmtree(d, ignore_errors=True)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--files", default=",".join(ORACLE_FILES))
    ap.add_argument("--jobs", type=int, default=8)
    ap.add_argument("--out", default=os.path.join(ROOT, "_build", "oracle_mutants.jsonl"))
    ap.add_argument("--rerun", default=None, help="only the survivors of this earlier output")
    ap.add_argument("--suites", default=",".join(PIN_SUITES), help="test files run against each mutant")
    args = ap.parse_args()
    suites = args.suites.split(",")
    workdir = os.path.join(ROOT, "_build", "oracle_mutants")
    trees, jobs = {}, []
    for rel in args.files.split(","):
        trees[rel] = ast.parse(open(os.path.join(ROOT, rel)).read())
        s = Sites()
        s.visit(trees[rel])
        jobs += [(rel, site) for site in s.sites]
    if args.rerun:
        keep = {(r["file"], r["kind"], r["index"]) for r in map(json.loads, open(args.rerun)) if not r["killed"]}
        jobs = [(rel, site) for rel, site in jobs if (rel, site[0], site[4]) in keep]
    print(len(jobs), "mutants", flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    killed = 0
    with open(args.out, "w") as out, ThreadPoolExecutor(args.jobs) as ex:
        futs = [ex.submit(_run_one, i, rel, trees[rel], site, workdir, suites) for i, (rel, site) in enumerate(jobs)]
        for f in futs:
            r = f.result()
            out.write(json.dumps(r) + "\n")
            out.flush()
            killed += r["killed"]
            if not r["killed"]:
                print("survived: %s:%d %s in %s" % (r["file"], r["line"], r["kind"], r["func"]), flush=True)
    print("%d of %d mutants killed" % (killed, len(jobs)))


if __name__ == "__main__":
    main()
