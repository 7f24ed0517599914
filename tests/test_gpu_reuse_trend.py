"""Image-quality trend of cross-view attribute reuse on the GPU (Eq. 6;
Table 1 trend), beside the FP64 oracle on the same crop.

Paper-scale mixture scene (200k Gaussians, 45 views, 4K panel), central
256x256 crop: for |V_k| = 1, 2, 4, 8 the GPU render must match the oracle
(bracket reading of the 1/255 threshold), and the PSNR of the |V_k| > 1 renders
against the exact |V_k| = 1 render must fall as |V_k| doubles, on the GPU as
in the oracle, with the two PSNRs close."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth

from .helpers import assert_render_matches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402


def psnr(a, b):
    mse = float(((np.clip(a, 0, 1) - np.clip(b, 0, 1)) ** 2).mean())
    return float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)


def test_reuse_trend_gpu_and_oracle():
    w = synth.WORKLOADS["paper4k"]
    scene = synth.scene_for(w, 200_000)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    V = oracle.view_index(w.panel)
    cx, cy = w.panel.width // 2, w.panel.height // 2
    crop = (cx - 128, cy - 128, cx + 128, cy + 128)
    ds = lfd.scene_to_device(scene)
    gpu, ref = {}, {}
    for c in (1, 2, 4, 8):
        plan = lfd.Plan(w.panel, tile=(32, 16), views_per_cluster=c)
        img, _ = plan.render(ds, cams)
        torch.cuda.synchronize()
        gpu[c] = img.cpu().numpy()[crop[1]:crop[3], crop[0]:crop[2]].astype(np.float64)
        plan.close()
        proj = oracle.project(scene, cams, w.panel.width, w.panel.height, c)
        ref[c], lo, hi = oracle.render_bracket(proj, V, c, crop=crop, mode=1)
        assert_render_matches(gpu[c], ref[c], lo, hi, what=f"|V_k|={c}")
    pg = [psnr(gpu[c], gpu[1]) for c in (2, 4, 8)]
    po = [psnr(ref[c], ref[1]) for c in (2, 4, 8)]
    for seq in (pg, po):
        assert seq[0] > seq[1] > seq[2], (pg, po)
    for a, b in zip(pg, po):
        assert abs(a - b) < 1.0, (pg, po)
