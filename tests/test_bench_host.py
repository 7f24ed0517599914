"""Host-side arithmetic of the benchmark line (no GPU)."""
import hashlib
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stage_rooflines_count_each_byte_once():
    # 1000 Gaussians of 236 B, K = 2 clusters of C = 4 views, P = 5000 pairs
    r = bench.stage_rooflines({"ms_project": 1.0, "ms_keygen": 2.0, "ms_sort": 4.0},
                              M=1000, K=2, C=4, P=5000, gaussian_bytes=236)
    proj = 2 * 1000 * (16 + 16 + 4 + 8 * 4)
    assert r["project"]["bytes"] == 1000 * 236 + proj
    assert r["keygen"]["bytes"] == proj + 5000 * 8
    assert r["sort"]["bytes"] == 5000 * 16
    assert r["sort"]["gbs"] == pytest.approx(5000 * 16 / 4e-3 / 1e9)
    assert r["project"]["frac"] == pytest.approx(r["project"]["gbs"] / r["peak_gbs"])


def test_hbm_peak_is_the_measured_copy_bandwidth_when_present():
    peak, which = bench.hbm_peak_gbs()
    assert peak > 0
    assert which in ("of measured", "of fallback")


def test_blend_traffic_only_for_the_captured_source_and_tile():
    path = os.path.join(ROOT, "profiles", "k_blend_traffic.txt")
    fields = dict(line.split(":", 1) for line in open(path) if ":" in line)
    tile = fields["tile"].strip()
    assert bench.blend_traffic_bytes("7x7") is None
    src = os.path.join(ROOT, "paper_2605_04509_gb300", "csrc", "blend.cu")
    current = hashlib.sha256(open(src, "rb").read()).hexdigest() == fields["blend_cu_sha256"].strip()
    want = int(fields["dram_bytes_per_launch"].strip()) if current else None
    assert bench.blend_traffic_bytes(tile) == want
