"""Host-side rules of bench.py that need no GPU: the DRAM traffic it reports comes from the committed ncu
record only while the kernel sources are the ones the counters were taken on, and is null otherwise."""
from __future__ import annotations

import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        return json.load(f)


def test_traffic_follows_the_recorded_sources(monkeypatch):
    rec = _record()
    for kernel in ("k_raster", "k_hq"):
        e = rec[kernel]["lidar100m"]
        monkeypatch.setattr(bench, "_csrc_digest", lambda e=e: e["csrc_digest"])
        assert bench._traffic(kernel, "lidar100m", 100) == e["bytes_per_point"] * 100
        # a traffic figure near the algorithmic 16 B per point: nothing is re-read
        assert 16.0 <= e["bytes_per_point"] < 17.5
        monkeypatch.setattr(bench, "_csrc_digest", lambda: "0" * 16)
        assert bench._traffic(kernel, "lidar100m", 100) is None
    assert bench._traffic("k_raster", "no-such-workload", 100) is None


def test_digest_covers_the_pass_kernels():
    d = bench._csrc_digest()
    assert len(d) == 16 and int(d, 16) >= 0
    assert d == bench._csrc_digest()


def test_traffic_only_for_the_captured_configuration(monkeypatch):
    """The record was taken on the exact transform with the default tuning: the other transforms and the
    random-order options run other kernels, so their lines carry no traffic figure."""
    import argparse
    e = _record()["k_hq"]["lidar100m"]
    monkeypatch.setattr(bench, "_csrc_digest", lambda: e["csrc_digest"])
    base = dict(transform="exact", band_filter=False, band_bounds=False)
    assert bench._traffic("k_hq", "lidar100m", 100, argparse.Namespace(**base)) == e["bytes_per_point"] * 100
    for change in (dict(transform="fp64"), dict(transform="double-float"), dict(band_filter=True),
                   dict(band_bounds=True)):
        assert bench._traffic("k_hq", "lidar100m", 100, argparse.Namespace(**{**base, **change})) is None


def test_digest_ignores_comments_and_layout():
    code = "int f(int a) {\n  return a + 1;  // one more\n}\n"
    same = "/* header */ int f(int a) { return a + 1; }"
    other = "int f(int a) { return a + 2; }"
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)
