"""Backward of the interlaced render against the FP64 autograd oracle
(oracle/torch_render.py, itself pinned against finite differences).

Setting of the differentiation workload, reduced to its check subset: 200
Gaussians, a 64x64 panel with 24 views (slant 0.2 rad, pitch 4.8), an L2 loss
to a target rendered from a copy whose means are perturbed by N(0, 0.01).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import torch_render
from paper_2605_04509_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402

KEYS = ("means", "scales", "quats", "opacities", "sh")


def case(c):
    panel = synth.Panel(64, 64, 24, math.tan(0.2), 4.8, 0.0)
    rig = synth.Rig(24, 40.0, 4.0, 50.0)
    scene = synth.uniform_scene(200, 5, half_extent=0.6)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    V = oracle.view_index(panel)
    rng = np.random.default_rng(6)
    moved = dict(scene)
    moved["means"] = (scene["means"] + rng.normal(0, 0.01, scene["means"].shape)).astype(np.float32)
    proj = oracle.project(moved, cams, panel.width, panel.height, c)
    target, _ = oracle.render(proj, V, c, mode=0)
    return panel, scene, cams, V, target


@pytest.mark.parametrize("c", [1, 8])
def test_gradients_match_fp64_autograd(c):
    panel, scene, cams, V, target = case(c)
    plan = lfd.Plan(panel, views_per_cluster=c)
    s = lfd.scene_to_device(scene)
    img, _ = plan.render(s, cams)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    grads = plan.backward(s, cams, 2.0 * (img - tgt))
    params = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in scene.items()}
    ref_img = torch_render.render(params, cams, V, c)
    loss = ((ref_img - torch.from_numpy(target)) ** 2).sum()
    loss.backward()
    for key in KEYS:
        got = grads[key].double().cpu().numpy().reshape(-1)
        ref = params[key].grad.numpy().reshape(-1)
        rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-12)
        cos = float(got @ ref / max(np.linalg.norm(got) * np.linalg.norm(ref), 1e-30))
        assert rel < 2e-2 and cos > 0.999, (key, rel, cos)
    plan.close()


def test_autograd_function_matches_entry_point():
    panel, scene, cams, V, target = case(8)
    plan = lfd.Plan(panel, views_per_cluster=8)
    s = lfd.scene_to_device(scene)
    leaves = {k: v.clone().requires_grad_(True) for k, v in s.items()}
    img = lfd.render_autograd(plan, cams, *(leaves[k] for k in KEYS))
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    ((img - tgt) ** 2).sum().backward()
    img2, _ = plan.render(s, cams)
    direct = plan.backward(s, cams, 2.0 * (img2 - tgt))
    for key in KEYS:
        assert torch.allclose(leaves[key].grad, direct[key], rtol=1e-5, atol=1e-7), key
    plan.close()
