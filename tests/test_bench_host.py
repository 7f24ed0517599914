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


def test_random_crops_in_bounds_with_both_corners():
    from paper_2605_04509_gb300 import synth
    panel = synth.WORKLOADS["paper4k"].panel
    crops = bench.random_crops(panel, 8, 128, seed=12)
    assert len(crops) == 8 and crops == bench.random_crops(panel, 8, 128, seed=12)
    assert crops[0] == (0, 0, 128, 128)
    assert crops[1] == (panel.width - 128, panel.height - 128, panel.width, panel.height)
    for x0, y0, x1, y1 in crops:
        assert 0 <= x0 and x1 <= panel.width and 0 <= y0 and y1 <= panel.height
        assert x1 - x0 == 128 and y1 - y0 == 128


def test_accuracy_verdicts_on_oracle_images():
    # the oracle's own image passes both readings; a planted error of 3e-3
    # away from any threshold jump fails both; a value inside a jump's span
    # fails only the literal bar
    import numpy as np

    import oracle
    from paper_2605_04509_gb300 import synth
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, 4)
    V = oracle.view_index(w.panel)
    crops = [(0, 0, 256, 144)]
    ref, lo, hi = oracle.render_bracket(proj, V, 4, mode=1)
    a = bench.accuracy_over_crops(ref.copy(), proj, V, 4, (16, 16), crops)
    assert a["bar_ok"] and a["literal_max_err_ok"] and a["max_err"] == 0.0
    span = np.maximum(np.maximum(ref, lo), hi) - np.minimum(np.minimum(ref, lo), hi)
    assert a["threshold_jump_subpixels"] == int((np.clip(span, 0, 1) > 1e-3).sum())
    quiet = np.argwhere((span == 0) & (ref > 0.1) & (ref < 0.9))[0]
    bad = ref.copy()
    bad[tuple(quiet)] += 3e-3
    b = bench.accuracy_over_crops(bad, proj, V, 4, (16, 16), crops)
    assert not b["bar_ok"] and not b["literal_max_err_ok"]
    jumps = np.argwhere((span > 3e-3) & (ref > 0.05) & (ref < 0.95))
    if len(jumps):
        j = tuple(jumps[0])
        other = ref.copy()
        other[j] = lo[j] if abs(lo[j] - ref[j]) > abs(hi[j] - ref[j]) else hi[j]
        c = bench.accuracy_over_crops(other, proj, V, 4, (16, 16), crops)
        assert c["bar_ok"] and not c["literal_max_err_ok"]
