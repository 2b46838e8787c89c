"""The benchmark's roofline arithmetic, on made-up solve statistics (no GPU):
the traversal's algorithmic bytes per launch with and without the stored
segment lists, the stored-segment product's 8 bytes per segment recovered
from the 7 it moves, and the DRAM-traffic figure, which is reported only for
the kernel source it was measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _trace_stats(hits, rays, nnz, trace_s, stored):
    return {"hits": hits, "rays": rays, "nnz": nnz, "trace_s": trace_s, "trace_launches": 1 if stored else 2,
            "segments_stored": 1 if stored else 0, "sphere_tests": 6 * hits, "node_visits": 2 * hits}


def test_traversal_that_stores_the_lists():
    # two steps, each one traversal of 1e6 rays that stored 3e7 entries for 2.9e7 hits,
    # 0.01 s per launch; each step's solve also ran a product (its rays are not the traversal's)
    st = [_trace_stats(2.9e7, 2e6, 3e7, 0.01, True) for _ in range(2)]
    r = bench.roofline(st, 2, 6800.0, "fallback", 1e6)
    per = 2.9e7 * 20 + 1e6 * 8 + 3e7 * 8
    assert r["alg_bytes_per_launch"] == pytest.approx(per)
    assert r["achieved"] == pytest.approx(per / 0.01 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["launch_ms"] == pytest.approx(10.0)
    assert r["hits_per_launch"] == pytest.approx(2.9e7) and r["rays_per_launch"] == pytest.approx(1e6)
    assert r["sphere_tests_per_hit"] == pytest.approx(6.0) and r["node_visits_per_hit"] == pytest.approx(2.0)
    assert r["peak_kind"] == "fallback" and r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_traversal_without_lists():
    # recomputed columns: two traversals per step, every ray's 4-byte column
    st = [_trace_stats(4e7, 2e6, 0, 0.03, False)]
    r = bench.roofline(st, 2, 6800.0, "measured", 1e6)
    per = (4e7 * 20 + 2e6 * 4) / 2
    assert r["alg_bytes_per_launch"] == pytest.approx(per)
    assert r["achieved"] == pytest.approx(per / 0.015 / 1e9)


def test_traffic_only_for_the_measured_source(monkeypatch):
    st = [_trace_stats(1e7, 1e6, 1.1e7, 0.01, True)]
    h = bench.source_hash("k_trace")
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "k_trace", {h: 12.5})
    assert bench.roofline(st, 1, 6800.0, "fallback", 1e6)["traffic"] == pytest.approx(12.5 * 1e7)
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "k_trace", {"0" * 16: 12.5})
    assert bench.roofline(st, 1, 6800.0, "fallback", 1e6)["traffic"] is None


def test_source_hash_is_per_kernel():
    # a fixed-length digest of the kernel's own source files
    a = bench.source_hash("k_trace")
    assert len(a) == 16 and a == bench.source_hash("k_trace")
    assert a != bench.source_hash("k_spmv")


def test_product_bytes_per_segment():
    # 3 launches over 1000 active particles (12 rays each): the product moved
    # 7 bytes per segment plus each ray's column and each particle's x
    n_act, launches, seg = 1000, 3, 5.0e6
    extra = launches * (n_act * 12 * 4 + n_act * 4)
    st = [{"spmv_launches": launches, "spmv_s": 0.003, "spmv_bytes": seg * 7 + extra, "n_active": n_act}]
    r = bench.roofline_spmv(st, 6800.0, "fallback")
    assert r["segments_per_launch"] == pytest.approx(seg / launches)
    per = (seg * 8 + extra) / launches
    assert r["alg_bytes_per_launch"] == pytest.approx(per)
    assert r["achieved"] == pytest.approx(per / 0.001 / 1e9)
