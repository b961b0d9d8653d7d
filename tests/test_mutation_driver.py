"""The mutation check of the oracle's pins (tests/oracle_mutation_sweep.py)
enumerates every +/- and unary-minus site, nested ones included, and each
mutant differs from the source in exactly the planted way."""
import ast
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle_mutation_sweep as M  # noqa: E402

SRC = "def f(a, b, c):\n    return a - b + (-c)\n"


def _mutants():
    tree = ast.parse(SRC)
    s = M.Sites()
    s.visit(tree)
    out = []
    for site in s.sites:
        m = M.Mutate(site[0], site[4])
        mutated = m.visit(ast.parse(SRC))
        assert m.done
        out.append((site[0], site[4], ast.unparse(ast.fix_missing_locations(mutated)).split("return ")[1]))
    return s.sites, out


def test_every_site_is_found_in_walk_order():
    sites, _ = _mutants()
    assert [(k, i) for k, _, _, _, i in sites] == [("swap", 0), ("dropr", 0), ("swap", 1), ("dropr", 1), ("neg", 2)]
    assert all(f == "f" for _, _, _, f, _ in sites)


def test_each_mutant_plants_exactly_one_mistake():
    _, out = _mutants()
    assert out == [("swap", 0, "a - b - -c"), ("dropr", 0, "a - b"),
                   ("swap", 1, "a + b + -c"), ("dropr", 1, "a + -c"), ("neg", 2, "a - b + c")]
