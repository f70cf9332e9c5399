"""Host-side helpers of bench.py (CPU): tile geometry, algorithmic bytes, the
traffic lookup and its source guard, the autotune cache, peaks and the job value."""
import json
import os

import pytest

import bench

N, P, NNZ = 500_000, 50_000, 114_693_671   # the bench workload


def test_tile_geometry_matches_the_captured_launches():
    """The tile and strip counts the ncu captures of the bench workload show
    (double-float values: 8 bytes; group width 1 and 2)."""
    assert bench.tile_geometry(N, P, 1, 8) == (2, 18)
    assert bench.tile_geometry(N, P, 2, 8) == (4, 36)
    assert bench.tile_geometry(N, P, 4, 8) == (8, 72)
    # float32 values hold twice the rows in the same 220 KB
    assert bench.tile_geometry(N, P, 1, 4) == (1, 9)


def test_bytes_per_launch_of_the_bench_products(monkeypatch):
    """Per RHS group at group width 2 (double-float): the figures quoted with
    the roofline (272.2 MB CSR, 273.6 MB CSC); the u kernel reads the T_c row
    partials and om and writes u."""
    monkeypatch.setattr(bench, "PRECISION", "df32")
    assert bench.bytes_per_launch("bt_csr_df32", N, P, NNZ, 16, 2) == pytest.approx(272.187346e6, rel=1e-9)
    assert bench.bytes_per_launch("bt_csc_df32", N, P, NNZ, 16, 2) == pytest.approx(273.587346e6, rel=1e-9)
    assert bench.bytes_per_launch("bt_u", N, P, NNZ, 16, 2) == 8 * 2 * (4 * N + 2 * N)
    # the fixed-point kernels move the same bytes as the double-float ones
    assert bench.bytes_per_launch("bt_csc_fx64", N, P, NNZ, 16, 2) == bench.bytes_per_launch(
        "bt_csc_df32", N, P, NNZ, 16, 2)
    assert bench.bytes_per_launch("bt_fin", N, P, NNZ, 16, 2) is None


def test_traffic_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"bt_csc_df32": {"source_sha": "abc",
                                                                   "dram_bytes_per_group": 1000}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "abc")
    assert bench.traffic_for("bt_csc_df32", 2.5) == 2500
    assert bench.traffic_for("bt_csr_df32", 2.5) is None        # not captured
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "changed")
    assert bench.traffic_for("bt_csc_df32", 2.5) is None        # kernels changed since the capture


def test_committed_traffic_matches_the_committed_kernels():
    """profiles/traffic.json was taken on the product kernels in the tree."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for k in ("bt_csr_df32", "bt_csc_df32"):
        assert d[k]["source_sha"] == bench.kernel_source_sha(), k


def test_tuned_group_width_reads_the_cache(tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("uneven:1:2 3\nbatch_rg:500000:50000:114693671:16:3 2\n")
    assert bench.tuned_group_width(str(f)) == 2
    assert bench.tuned_group_width(str(tmp_path / "missing.txt")) == 1


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6768.1}))
    assert bench.peaks() == (6768.1, "measured")


def test_job_value_counts_every_rank():
    assert bench.job_value(1, 2000.0) == pytest.approx(bench.NRHS / 2.0)
    assert bench.job_value(4, 2000.0) == pytest.approx(4 * bench.NRHS / 2.0)
