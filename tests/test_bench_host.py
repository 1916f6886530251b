"""Host-side parts of bench.py (no GPU): the algorithmic work table against the oracle's counters, and the
flop and roofline arithmetic built on it."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_work_table_row_matches_the_oracle():
    # the 4096-point row, re-derived from the oracle's counters on the same 2048-cell sample
    import work_per_cell

    c = work_per_cell.counters("uniform4096", 2048)
    row = bench.WORK["uniform4096"]
    for k in ("n_cert", "verts", "faces"):
        assert abs(c[k] - row[k]) <= 0.005 + 1e-9, (k, c[k], row[k])


def test_work_counters_match_poisson_means():
    # uniform points: the final cells are Poisson-Voronoi cells, whose mean vertex and facet counts are
    # 96 pi^2 / 35 and 2 + 48 pi^2 / 35 (Meijering); the 2048-cell sample is within a few standard errors
    import math

    row = bench.WORK["uniform4096"]
    assert abs(row["verts"] - 96 * math.pi ** 2 / 35) < 0.3
    assert abs(row["faces"] - (2 + 48 * math.pi ** 2 / 35)) < 0.15


def test_flops_per_cell_formula():
    w = {"n_cert": 10.0, "verts": 2.0, "faces": 3.0}
    assert bench.flops_per_cell(w) == 10 * 2 * 6 + 2 * 40 + 3 * 30
    assert bench.flops_per_cell(bench.WORK["clustered16M"]) == pytest.approx(27_700, rel=0.01)


def test_step_roofline_takes_the_larger_bound_per_stage():
    N, G, faces = 1000, 0, 15.0
    clip_bytes = 32 * faces + 40
    per_cell = 24 + 6 * 32 + 40 + clip_bytes + (36 * faces + 8) + 40 + (40 * faces + 12) + (36 * faces + 12)
    ms_per_byte = 1e3 / (bench.HBM_GBS * 1e9)
    # clipping bound by its flops: the clipping bytes drop out of the sum
    fpc = 1e9
    r = bench.step_roofline(N, G, faces, fpc, 1.0, 10.0)
    t_alu = fpc * N / 1e12 * 1e3
    assert r["bytes_per_cell"] == per_cell
    assert r["t_roof_ms"] == pytest.approx((per_cell - clip_bytes) * N * ms_per_byte + t_alu, rel=1e-12)
    assert r["frac"] == pytest.approx(r["t_roof_ms"] / 10.0)
    # no flops: every stage bound by its bytes, grid nodes included
    r = bench.step_roofline(N, 8, faces, 0.0, 1.0, 10.0)
    assert r["t_roof_ms"] == pytest.approx((per_cell * N + 4 * 8 ** 3) * ms_per_byte, rel=1e-12)


def test_clock_samples_summary():
    lines = ["0, 2070, 2070, 1012.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1965, 2070, 1398.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, [N/A], 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbled line",
             "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    r = bench.Clocks.summarise(lines)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = ["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active"] * 2
    r = bench.Clocks.summarise(hot)
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0
    assert bench.Clocks.summarise([])["sm_mhz"] is None


def test_workload_cache_is_keyed_by_the_generator(monkeypatch, tmp_path):
    # the cached point set is reused only for the same generator source
    import tempfile

    monkeypatch.setattr(tempfile, "gettempdir", lambda: str(tmp_path))
    x1, d1 = bench.workload("uniform4096")
    files = sorted(p.name for p in tmp_path.iterdir())
    assert files == ["vt_bench_uniform4096_%s.npy" % bench._inputs_tag()]
    x2, _ = bench.workload("uniform4096")  # from the cache
    assert (x1 == x2).all() and d1["N"] == 4096 == len(x1)
    monkeypatch.setattr(bench, "_inputs_tag", lambda: "0123456789")
    bench.workload("uniform4096")
    assert len(list(tmp_path.iterdir())) == 2


def test_both_arms_describe_the_same_workload():
    x, desc = bench.workload("uniform4096")
    c = bench.workload_config(desc, 1)
    assert c == {"workload": desc["workload"], "grid": "32^3", "parallelism": "1 GPU"}
    assert bench.workload_config(dict(desc, grid=0), 2)["grid"].startswith("none")
    assert bench.workload_config(desc, 2)["parallelism"] == "replicas"


def test_hbm_peak_comes_from_the_measured_peaks_file(monkeypatch, tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 1234.5}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._hbm_gbs() == 1234.5
    (tmp_path / "MEASURED_PEAKS.json").write_text("not json")
    assert bench._hbm_gbs(default=7.0) == 7.0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench._hbm_gbs(default=8.0) == 8.0


def test_alu_peaks_from_unit_counts():
    # 152 SMs at 2070 MHz: 128 FP32 lanes -> 80.5 TFLOP/s; the FP64 pipe is 1/64 of it
    p32, p64 = bench.alu_peaks(152, 2070.0)
    assert p32 == pytest.approx(80.54784)
    assert p64 == pytest.approx(p32 / 64)


def test_oracle_timer_rates_cells_without_the_tree():
    """The CPU baseline's oracle builds its tree once, outside the timed sample, and reports both."""
    from paper_1601_06429_gb300 import inputs

    x = inputs.uniform(4096, seed=0, dtype=np.float32)
    t = bench.OracleTimer(x, {"L": 1.0, "N": len(x)})
    r, info = t.rate(512, seed=1)
    assert r > 0 and info["tree_seconds"] == t.tree_seconds >= 0 and "512 random cells" in info["sample"]
    pts, off = inputs.halo_sets(n_sets=3, nmin=100, nmax=400, seed=6)
    ts = bench.OracleTimer(pts, {"set_off": off, "N": len(pts)})
    r, info = ts.rate(64, seed=2)
    assert r > 0 and len(ts.trees) == 3


def test_parity_report_of_oracle_outputs_is_exact():
    """The bench's per-output error report, fed outputs computed by the oracle itself (brute force): zero
    errors, identical neighbour lists; a perturbed volume shows up as its relative error."""
    import oracle
    from paper_1601_06429_gb300 import inputs

    x = inputs.uniform(1024, seed=5)
    o = oracle.cells(x, 0.0, 1.0, True, mode="brute")
    off, ids = oracle.neighbours(o)
    dens = 1.0 / o["vol"]
    noff, nids, disp = oracle.neighbour_displacements(o, x, 0.0, 1.0)
    grad = oracle.gradient(dens, noff, nids, disp, dens)
    out = dict(vol=o["vol"].copy(), dens=dens, grad=grad, off=off, ids=ids)
    flags = np.zeros(len(x), np.uint8)
    flags[7] = 2
    tree = oracle.Tree(x, 0.0, 1.0, True)
    r = bench.parity_report(x, 1.0, tree, out, flags, n_sample=300, n_grad=40)
    assert r["nbr_lists_different"] == 0 and r["exact_cells"] == 1
    assert r["vol_max_rel"] < 1e-14 and r["dens_max_rel"] < 1e-14 and r["grad_max_err_floor_1e-3"] < 1e-9
    out["vol"][7] *= 1 + 3e-6
    assert bench.parity_report(x, 1.0, tree, out, flags, n_sample=300, n_grad=40)["vol_max_rel"] == \
        pytest.approx(3e-6, rel=1e-6)
