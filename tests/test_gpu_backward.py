"""Backward of the interlaced render against the FP64 autograd oracle
(oracle/torch_render.py, itself pinned against finite differences).

Setting of the differentiation workload, reduced to its check subset: 200
Gaussians, a 64x64 panel with 24 views (slant 0.2 rad, pitch 4.8), an L2 loss
to a target rendered from a copy whose means are perturbed by N(0, 0.01).
Both backward forms are covered: from the blend state kept by the forward
frame, and re-blending the lists. Clusters of 24 views give runs longer than
a block (processed in chunks); the 45-view panel (pitch 4.6) puts two or
three views in one warp.
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


def case(c, views=24, pitch=4.8):
    panel = synth.Panel(64, 64, views, math.tan(0.2), pitch, 0.0)
    rig = synth.Rig(views, 40.0, 4.0, 50.0)
    scene = synth.uniform_scene(200, 5, half_extent=0.6)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    V = oracle.view_index(panel)
    rng = np.random.default_rng(6)
    moved = dict(scene)
    moved["means"] = (scene["means"] + rng.normal(0, 0.01, scene["means"].shape)).astype(np.float32)
    proj = oracle.project(moved, cams, panel.width, panel.height, c)
    target, _ = oracle.render(proj, V, c, mode=0)
    return panel, scene, cams, V, target


def check_against_oracle(c, kept, views=24, pitch=4.8):
    panel, scene, cams, V, target = case(c, views, pitch)
    plan = lfd.Plan(panel, views_per_cluster=c)
    if kept:
        plan.set_flags(lfd.FLAG_KEEP_BLEND_STATE)
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


@pytest.mark.parametrize("kept", [False, True])
@pytest.mark.parametrize("c", [1, 8, 24])
def test_gradients_match_fp64_autograd(c, kept):
    check_against_oracle(c, kept)


@pytest.mark.parametrize("kept", [False, True])
def test_gradients_match_fp64_autograd_several_views_per_warp(kept):
    check_against_oracle(8, kept, views=45, pitch=4.6)


def test_kept_state_matches_replay():
    panel, scene, cams, V, target = case(8)
    s = lfd.scene_to_device(scene)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    out = []
    for kept in (False, True):
        plan = lfd.Plan(panel, views_per_cluster=8)
        if kept:
            plan.set_flags(lfd.FLAG_KEEP_BLEND_STATE)
        img, _ = plan.render(s, cams)
        out.append((img.clone(), plan.backward(s, cams, 2.0 * (img - tgt))))
        plan.close()
    # the kept state leaves the image bit-identical; the gradients differ
    # only by the order of the floating-point atomics that sum them
    assert torch.equal(out[0][0], out[1][0])
    for key in KEYS:
        err = float((out[0][1][key] - out[1][1][key]).abs().max())
        scale = float(out[0][1][key].abs().max())
        assert err <= 1e-4 * scale, (key, err, scale)


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
    # the gradients are summed with floating-point atomics, whose order varies
    # from run to run: compare against the gradient's own scale
    for key in KEYS:
        err = float((leaves[key].grad - direct[key]).abs().max())
        scale = float(direct[key].abs().max())
        assert err <= 1e-4 * scale, (key, err, scale)
    plan.close()


def test_kept_state_in_capacity_mode_under_graph():
    # the kept blend state is allocated by set_flags, so capacity-mode frames
    # (no host read-back, no allocation) keep it inside a captured graph too
    panel, scene, cams, V, target = case(8)
    s = lfd.scene_to_device(scene)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    ref_plan = lfd.Plan(panel, views_per_cluster=8)
    ref_plan.set_flags(lfd.FLAG_KEEP_BLEND_STATE)
    want, st = ref_plan.render(s, cams)
    want = want.clone()
    ref = ref_plan.backward(s, cams, 2.0 * (want - tgt))
    plan = lfd.Plan(panel, views_per_cluster=8)
    plan.set_flags(lfd.FLAG_KEEP_BLEND_STATE)
    plan.reserve(s["means"].shape[0], 2 * int(st["num_pairs"]) + 16)
    out = torch.zeros_like(want)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.render(s, cams, out=out)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.render(s, cams, out=out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert plan.status() == int(st["num_pairs"])
    assert torch.equal(out, want)
    got = plan.backward(s, cams, 2.0 * (out - tgt))
    for key in KEYS:
        err = float((got[key] - ref[key]).abs().max())
        scale = float(ref[key].abs().max())
        assert err <= 1e-4 * scale, (key, err, scale)
    plan.close()
    ref_plan.close()
