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


N5, P5, NNZ5 = 500_000, 50_000, 114_693_671


def write_traffic(tmp_path, monkeypatch, entry):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"bt_csc_df32": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "abc")


def test_traffic_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    write_traffic(tmp_path, monkeypatch, {"source_sha": "abc", "rhs_group": 2, "live_chains": 16,
                                          "dram_bytes_per_launch": 1000, "smem_wavefronts_per_launch": 160})
    full = bench.scope_table_bytes("bt_csc_df32", N5, P5, NNZ5, 16)
    assert bench.traffic_for("bt_csc_df32", full, N5, P5, NNZ5, 2) == pytest.approx(1000)
    assert bench.traffic_for("bt_csr_df32", full, N5, P5, NNZ5, 2) is None       # not captured
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "changed")
    assert bench.traffic_for("bt_csc_df32", full, N5, P5, NNZ5, 2) is None       # kernels changed


def test_traffic_scales_with_the_launch_and_group_width(tmp_path, monkeypatch):
    """A launch with fewer live chains moves fewer algorithmic bytes and
    gathers fewer entries; a capture at another group width is not used."""
    write_traffic(tmp_path, monkeypatch, {"source_sha": "abc", "rhs_group": 2, "live_chains": 16,
                                          "dram_bytes_per_launch": 1000, "smem_wavefronts_per_launch": 160})
    half = bench.scope_table_bytes("bt_csc_df32", N5, P5, NNZ5, 8)
    full = bench.scope_table_bytes("bt_csc_df32", N5, P5, NNZ5, 16)
    assert bench.traffic_for("bt_csc_df32", half, N5, P5, NNZ5, 2) == pytest.approx(1000 * half / full)
    assert bench.smem_wavefronts_for("bt_csc_df32", 8, 2) == pytest.approx(80)
    assert bench.traffic_for("bt_csc_df32", full, N5, P5, NNZ5, 8) is None       # captured at RG = 2
    assert bench.smem_wavefronts_for("bt_csc_df32", 8, 8) is None


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


def test_product_accounting_splits_main_and_tail_plans():
    """Chains of 3, 1 and 5 iterations at group width 2 with a tail plan:
    live counts 3, 2, 2, 1, 1 per iteration; the main plan works in the three
    iterations with two or more chains (groups 2 + 1 + 1, chains 3 + 2 + 2)
    and the tail plan in the last two."""
    a = bench.product_accounting([3, 1, 5], 2, tail=True)
    assert a == {"iterations": 5, "main_iterations": 3, "tail_iterations": 2,
                 "main_group_units": 4, "main_chain_units": 7, "tail_chain_units": 2,
                 "main_slot_units": 4 + 2 + 2, "tail_slots": 2}
    b = bench.product_accounting([3, 1, 5], 2, tail=False)
    assert b["main_iterations"] == 5 and b["main_group_units"] == 6 and b["tail_iterations"] == 0


def test_scope_table_bytes_share_the_index_streams():
    """The scope table's bytes: one CSC pass over 16 chains reads the 4-byte
    row indices once, each chain's vectors once: about 1.04 GB for the two
    product passes of one 16-chain iteration (the table's 1.09 GB per
    iteration adds the CG update's vectors)."""
    one = bench.scope_table_bytes("bt_csc_df32", N, P, NNZ, 1)
    sixteen = bench.scope_table_bytes("bt_csc_df32", N, P, NNZ, 16)
    assert one == 4 * NNZ + 8 * (P + 1) + 4 * N + 24 * P
    assert sixteen - one == 15 * (4 * N + 24 * P)
    both = sixteen + bench.scope_table_bytes("bt_csr_df32", N, P, NNZ, 16)
    assert 1.03e9 < both < 1.05e9


def test_roofline_counts_only_working_launches():
    """A profile where the main CSC kernel ran 5 launches (3 working, 2 at its
    gate) for 6 ms: achieved = scope-table bytes of the 3 working launches
    over the 6 ms, and avg_launch_us = 6 ms / 3."""
    acct = bench.product_accounting([3, 1, 5], 2, tail=True)
    table = {"bt_csc_df32": (6.0, 5), "bt1_csc_df32": (1.0, 5), "b_update": (0.5, 5)}
    r = bench.roofline(table, acct, N, P, NNZ, 2, 6800.0, "measured")
    want = (3 * (4 * NNZ + 8 * (P + 1)) + 7 * (4 * N + 24 * P)) / 6e-3 / 1e9
    assert r["kernel"] == "bt_csc_df32" and r["working_launches"] == 3
    assert r["achieved"] == pytest.approx(want) and r["frac"] == pytest.approx(want / 6800.0)
    assert r["avg_launch_us"] == pytest.approx(2000.0)
    assert r["per_kernel"]["bt1_csc_df32"]["working_launches"] == 2


def test_projected_rate_arithmetic(monkeypatch):
    """Whole draws projected from (rhs seconds, seconds per iteration): two
    chains of 10 and 30 iterations on one thread take 1 + 10 + 2 + 60 = 73 s."""
    monkeypatch.setattr(bench, "oracle_iters", lambda P, r, g=None: ([10, 30][r], "test"))
    rate, _ = bench.projected_rate([(0, 1.0, 1.0), (1, 2.0, 2.0)], 1, None)
    assert rate == pytest.approx(2 / 73.0)
    rate2, _ = bench.projected_rate([(0, 1.0, 1.0), (1, 2.0, 2.0)], 2, None)
    assert rate2 == pytest.approx(2 / 36.5)


def test_shared_wavefronts_follow_the_same_source_guard(tmp_path, monkeypatch):
    write_traffic(tmp_path, monkeypatch, {"source_sha": "abc", "live_chains": 16,
                                          "dram_bytes_per_launch": 1000, "smem_wavefronts_per_launch": 320})
    assert bench.smem_wavefronts_for("bt_csc_df32", 4.0) == pytest.approx(80)
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "changed")
    assert bench.smem_wavefronts_for("bt_csc_df32", 4.0) is None


def test_finalize_bytes_follow_the_covered_slots(monkeypatch):
    """k_b_fin reads the strip partials of the slots it covers (4, 2, 2 in
    the three main iterations of chains 3, 1, 5 at group width 2) and, in
    the two tail iterations, the one chain's partials over the width-1
    strips; s, d and v are 24 bytes per covered slot and column."""
    monkeypatch.setattr(bench, "PRECISION", "df32")
    acct = bench.product_accounting([3, 1, 5], 2, tail=True)
    table = {"bt_csc_df32": (6.0, 5), "bt_fin": (1.0, 5)}
    r = bench.roofline(table, acct, N, P, NNZ, 2, 6800.0, "measured")
    T2, T1 = bench.tile_geometry(N, P, 2, 8)[1], bench.tile_geometry(N, P, 1, 8)[1]
    want = P * (8 * (8 * T2 + 24) + 2 * (8 * T1 + 24 * 2))
    assert r["per_kernel"]["bt_fin"]["impl_GBps"] == pytest.approx(want / 1e-3 / 1e9, rel=1e-3)
