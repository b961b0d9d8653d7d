"""Host-side bookkeeping of bench.py (no GPU): the algorithmic stage bytes of
a step scale with the number of points, exceed the compulsory bytes, are
smaller in the mixed-precision leg (FP32 stencil fields), and the stored
traffic constants are refused for another grid."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def _sizes(b):
    nc = 80 * 4 ** b
    return nc, 3 * nc // 2, nc // 2 + 2


def test_stage_bytes_scale_and_order():
    B = _bench()
    for nlev in (30, 90):
        s5 = B.stage_bytes_per_step("fp64", *_sizes(5), nlev, 5)
        s6 = B.stage_bytes_per_step("fp64", *_sizes(6), nlev, 5)
        assert abs(s6 / s5 - 4.0) < 1e-3          # linear in the points (2 more vertices per grid)
        m6 = B.stage_bytes_per_step("mixed", *_sizes(6), nlev, 5)
        assert m6 < s6
        nc, ne, nv = _sizes(6)
        assert s6 > B.compulsory_bytes_per_step(nc, ne, nlev, 5)
    assert B.stage_bytes_per_step("learned", *_sizes(6), 90, 5) is None


def test_traffic_constants_only_for_the_captured_grid():
    B = _bench()
    saved = dict(B.WORKLOAD)
    try:
        B.WORKLOAD["bisections"] = 5
        assert B.column_traffic() is None
        assert B.dram_measured("fp64", 100.0) is None
    finally:
        B.WORKLOAD.clear()
        B.WORKLOAD.update(saved)
