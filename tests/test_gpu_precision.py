"""FP16 / BF16 attribute storage on the 8K / 100-view precision panel,
against the FP64 oracle.

The kernel error is taken against the oracle fed the dequantised attributes
(every FP16 / BF16 value is exact in FP32 and FP64) and must meet the bar
(max |err| <= 2e-3 outside the 1/255 threshold jumps, <= 0.1 % of subpixels
off by more than 1/255). The storage error against the oracle on the FP32
originals is printed and only bounded loosely. Sampled size: 1M of the
workload's 3M Gaussians (the oracle projects every Gaussian into all 100
views) and the central 256x256 crop.
"""
import json

import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth

from .helpers import assert_render_matches, image_metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402

M = 1_000_000
CROP = 256


@pytest.fixture(scope="module")
def case():
    w = synth.WORKLOADS["precision8k"]
    scene = synth.scene_for(w, M)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    x0, y0 = (w.panel.width - CROP) // 2, (w.panel.height - CROP) // 2
    crop = (x0, y0, x0 + CROP, y0 + CROP)
    V = oracle.view_index(w.panel)
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, 8)
    ref32, _ = oracle.render(proj, V, 8, crop=crop, mode=1, tile=(32, 16))
    return w, scene, cams, crop, V, ref32


@pytest.mark.parametrize("dt", ["float16", "bfloat16"])
def test_half_attributes_on_8k_panel(case, dt):
    w, scene, cams, crop, V, ref32 = case
    plan = lfd.Plan(w.panel, tile=(32, 16), views_per_cluster=8)
    s = lfd.scene_to_device(scene, attr_dtype=getattr(torch, dt))
    img, _ = plan.render(s, cams)
    got = img[crop[1]:crop[3], crop[0]:crop[2]].cpu().numpy()
    deq = {k: v.float().cpu().numpy() for k, v in s.items()}
    proj = oracle.project(deq, cams, w.panel.width, w.panel.height, 8)
    ref, lo, hi = oracle.render_bracket(proj, V, 8, crop=crop, mode=1, tile=(32, 16))
    kernel = assert_render_matches(got, ref, lo, hi, f"{dt} attributes, 8K crop")
    storage = image_metrics(got, ref32)
    print(json.dumps({"attributes": dt, "crop": list(crop), "gaussians": M,
                      "vs_dequantised_oracle": kernel, "vs_fp32_oracle": storage}))
    assert storage["psnr"] > 35
    plan.close()
