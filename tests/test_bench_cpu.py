"""Host-side bookkeeping of bench.py (no GPU): the algorithmic stage bytes of
a step scale with the number of points, exceed the compulsory bytes, are
smaller in the mixed-precision leg (FP32 stencil fields); the per-unit DRAM
figures of the one-kernel captures are scaled by units and launches, and
refused once the kernel sources or the level count differ."""
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


def test_kernel_names_map_to_their_base_kernel_and_units():
    B = _bench()
    nc, ne, nv = _sizes(5)
    for name in ("sn_column_corr_terrain_mx64", "sn_column_corr_mx", "sn_column_corr_terrain", "sn_column_corr"):
        assert B.base_name(name) == "sn_column_corr"
        assert B.units_per_launch(name, nc, ne, nv, 90) == nc * 90
    assert B.base_name("va_edge_tend_terrain_f32") == "va_edge_tend"
    assert B.units_per_launch("va_edge_tend_terrain_f32", nc, ne, nv, 90) == ne * 91
    assert B.units_per_launch("va_concorr", nc, ne, nv, 90) == nc * 91


def _with_table(B, table):
    saved = dict(B.DRAM_PER_UNIT)
    B.DRAM_PER_UNIT.update(table)
    return saved


def test_dram_figures_only_for_the_captured_sources_and_levels():
    B = _bench()
    saved = _with_table(B, {"sources_sha256": B.sources_sha256(), "nlev": 90,
                            "legs": {"fp64": {"sn_column_pred": 100.0, "va_edge_tend": 50.0}}})
    try:
        assert B.dram_table("fp64", 90) is not None
        assert B.dram_table("fp64", 65) is None            # another level count
        assert B.dram_table("mixed", 90) is None           # a leg not captured
        B.DRAM_PER_UNIT["sources_sha256"] = "0" * 64       # the kernels changed since the capture
        assert B.dram_table("fp64", 90) is None
    finally:
        B.DRAM_PER_UNIT.clear()
        B.DRAM_PER_UNIT.update(saved)


def test_dram_arithmetic_scales_per_unit_bytes_by_units_and_launches():
    B = _bench()
    nc, ne, nv = _sizes(6)
    saved = _with_table(B, {"sources_sha256": B.sources_sha256(), "nlev": 90,
                            "legs": {"fp64": {"sn_column_pred": 100.0, "va_edge_tend": 50.0}}})
    try:
        prof = {"sn_column_pred": (10, 20.0), "va_edge_tend": (40, 10.0)}
        r = B.dram_measured("fp64", prof, 2, 100.0, (nc, ne, nv), 90, 5)
        b = (100.0 * nc * 90 * 10 + 50.0 * ne * 91 * 40) / 2
        assert abs(r["bytes_per_step"] - b) < 1e-6 * b
        assert abs(r["achieved_gbs"] - b / 0.1 / 1e9) < 1e-9 * r["achieved_gbs"]
        assert abs(r["frac"] - r["achieved_gbs"] / B.hbm_peak()[0]) < 1e-15
        prof["sn_cell_grad"] = (5, 1.0)                    # a kernel without a captured figure
        assert B.dram_measured("fp64", prof, 2, 100.0, (nc, ne, nv), 90, 5) is None
        # the roofline's dominant family carries its own traffic and HBM fraction
        r = B.roofline({"sn_column_pred": (5, 10.0), "sn_column_corr": (5, 12.0)}, nc, ne, nv, 90)
        assert r["traffic"] is None                        # the corrector form was not captured
        B.DRAM_PER_UNIT["legs"]["fp64"]["sn_column_corr"] = 140.0
        r = B.roofline({"sn_column_pred": (5, 10.0), "sn_column_corr": (5, 12.0)}, nc, ne, nv, 90)
        per = (100.0 + 140.0) * nc * 90 * 5
        assert abs(r["traffic"] - per / 10) < 1e-6 * per
        assert abs(r["hbm"]["achieved_gbs"] - per / 0.022 / 1e9) < 1e-9 * r["hbm"]["achieved_gbs"]
    finally:
        B.DRAM_PER_UNIT.clear()
        B.DRAM_PER_UNIT.update(saved)


def test_roofline_takes_the_longest_family_and_counts_its_flops():
    """The column solve's predictor and corrector form one family; with the
    longest summed time it is the one reported, at (the two forms' flops per
    column-level) x columns x levels x launches over its summed time."""
    B = _bench()
    nc, ne, nv = _sizes(6)
    nlev = 90
    prof = {"sn_column_pred": (5, 10.0), "sn_column_corr": (5, 12.0), "va_edge_tend": (10, 15.0)}
    r = B.roofline(prof, nc, ne, nv, nlev)
    flops = (B.FLOPS_PER_UNIT["sn_column_pred"] + B.FLOPS_PER_UNIT["sn_column_corr"]) * nc * nlev * 5
    assert r["kernel"] == "sn_column" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - flops / 0.022 / 1e12) < 1e-12 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / B.FP64_PEAK_TFLOPS) < 1e-15
    # a larger edge-tendency time moves the report to that kernel, at its flops per edge-half-level
    prof["va_edge_tend"] = (10, 30.0)
    r = B.roofline(prof, nc, ne, nv, nlev)
    assert r["kernel"] == "va_edge_tend"
    tab = B.dram_table("fp64", nlev)
    if tab is None:   # no capture of the running sources: no traffic figure
        assert r["traffic"] is None
    else:             # the captured bytes per unit times the units of one launch
        want = tab["va_edge_tend"] * ne * (nlev + 1)
        assert abs(r["traffic"] - want) < 1e-9 * want and r["hbm"]["achieved_gbs"] > 0
    f = B.FLOPS_PER_UNIT["va_edge_tend"]
    assert abs(r["achieved"] - f * ne * (nlev + 1) * 10 / 0.030 / 1e12) < 1e-12 * r["achieved"]


def test_kernel_table_per_step_and_shares():
    B = _bench()
    t = B.kernel_table({"a": (10, 30.0), "b": (4, 10.0)}, 2)
    assert list(t) == ["a", "b"]
    assert t["a"] == {"launches_per_step": 5, "ms_per_step": 15.0, "share": 0.75}
    assert t["b"] == {"launches_per_step": 2, "ms_per_step": 5.0, "share": 0.25}


def test_cpu_sample_scaled_to_a_full_step():
    """A sample of one substep and one diffusion on 1/16 of the columns: a
    full step is 16 x (ndyn substeps + diffusion)."""
    B = _bench()
    assert abs(B.sample_to_steps_per_s(1.6, 0.4, 16) - 1.0 / (16 * (5 * 1.6 + 0.4))) < 1e-15


def test_state_and_compulsory_bytes_are_those_of_the_state_arrays():
    """The six prognostic arrays (vn, w, rho, exner, theta_v, exner_pr) as the
    inputs give them: state_bytes is their total size, and the compulsory
    traffic reads and writes them once per substep and once for diffusion."""
    B = _bench()
    import numpy as np
    from icon_inputs import make_grid, make_vct, jw_type_state
    grid, z = make_grid(1), make_vct(12)
    st = jw_type_state(grid, z)
    st["exner_pr"] = np.zeros_like(st["exner"])
    total = sum(np.ascontiguousarray(st[k], dtype=np.float64).nbytes
                for k in ("vn", "w", "rho", "exner", "theta_v", "exner_pr"))
    assert B.state_bytes(grid.n_cells, grid.n_edges, 12) == total
    assert B.compulsory_bytes_per_step(grid.n_cells, grid.n_edges, 12, 5) == 2 * 6 * total


def test_chunked_kernels_count_their_bytes_per_step():
    """The learned step's networks and increments run in row chunks: their
    captured bytes are per unit of a whole step (cells for the GEMMs), so
    the number of chunk launches does not multiply them."""
    B = _bench()
    nc, ne, nv = _sizes(6)
    nlev = 90
    table = {"mlp_gemm_tc": 1000.0, "lc_apply_col": 2.0, "va_edge_pre_f32": 3.0, "va_edge_pre": 3.0}
    saved = _with_table(B, {"sources_sha256": B.sources_sha256(), "nlev": 90, "legs": {"learned": table}})
    try:
        for chunks in (1, 4):
            prof = {"mlp_gemm_tc": (3 * chunks, 1.0), "lc_apply_col": (chunks, 1.0), "va_edge_pre_f32": (6, 1.0)}
            r = B.dram_measured("learned", prof, 1, 10.0, (nc, ne, nv), nlev, 3)
            want = 1000.0 * nc + 2.0 * nc * (3 * nlev - 1) + 3.0 * ne * nlev * 6
            assert abs(r["bytes_per_step"] - want) < 1e-9 * want
    finally:
        B.DRAM_PER_UNIT.clear()
        B.DRAM_PER_UNIT.update(saved)
