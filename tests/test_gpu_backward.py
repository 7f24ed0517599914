"""Backward of the interlaced render against the FP64 autograd oracle
(oracle/torch_render.py, itself pinned against finite differences), entry by
entry, and against finite differences of the FP64 oracle loss directly.

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


def oracle_grads(scene, cams, V, c, target, alpha_min=torch_render.ALPHA_MIN):
    """FP64 autograd gradient of the L2 loss to the target."""
    params = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in scene.items()}
    img = torch_render.render(params, cams, V, c, alpha_min=alpha_min)
    ((img - torch.from_numpy(target)) ** 2).sum().backward()
    return {k: params[k].grad.numpy().reshape(-1) for k in KEYS}


# Element-wise bound on each gradient entry g against the FP64 reference r:
# |g - r| <= ATOL_REL * max|r| + RTOL * |r|. FP32 evaluation of the forward
# quantities (relative ~1e-6 each) and FP32 atomic sums over up to a few
# thousand subpixel contributions keep the error far below RTOL for the
# large entries; ATOL_REL covers entries whose contributions cancel.
ATOL_REL, RTOL = 1e-3, 1e-2


def check_against_oracle(c, kept, views=24, pitch=4.8):
    panel, scene, cams, V, target = case(c, views, pitch)
    plan = lfd.Plan(panel, views_per_cluster=c)
    if kept:
        plan.set_flags(lfd.FLAG_KEEP_BLEND_STATE)
    s = lfd.scene_to_device(scene)
    img, _ = plan.render(s, cams)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    grads = plan.backward(s, cams, 2.0 * (img - tgt))
    # the reference, and the same with the 1/255 skip threshold moved by
    # -/+0.1 %: where a Gaussian's alpha sits at the threshold, FP32 may skip
    # it where FP64 does not (or the reverse), which changes the gradient by
    # that Gaussian's whole contribution; such entries must lie within the
    # span of the three references (the accuracy reading of the render)
    ref = oracle_grads(scene, cams, V, c, target)
    lo = oracle_grads(scene, cams, V, c, target, torch_render.ALPHA_MIN * (1 - 1e-3))
    hi = oracle_grads(scene, cams, V, c, target, torch_render.ALPHA_MIN * (1 + 1e-3))
    for key in KEYS:
        got = grads[key].double().cpu().numpy().reshape(-1)
        r = ref[key]
        low = np.minimum(np.minimum(r, lo[key]), hi[key])
        high = np.maximum(np.maximum(r, lo[key]), hi[key])
        tol = ATOL_REL * max(float(np.abs(r).max()), 1e-30) + RTOL * np.abs(r)
        dist = np.abs(got - np.clip(got, low, high))
        worst = int(np.argmax(dist - tol))
        assert (dist <= tol).all(), (key, int((dist > tol).sum()), "worst", worst, got[worst], r[worst],
                                     low[worst], high[worst], tol[worst])
        # the bracket only widens the bound where the threshold moves the
        # reference; elsewhere the plain element-wise bound holds
        plain = np.abs(got - r) <= tol
        assert plain.mean() >= 0.995, (key, float(plain.mean()))
    plan.close()


def test_gradients_match_fp64_finite_differences():
    """The GPU gradient against central finite differences of the FP64 oracle
    loss, on the entries with the largest GPU gradient (six per parameter
    group). The step is small enough that no subpixel crosses the 1/255 or
    T thresholds: entries whose differences at step h and 2h disagree are
    skipped, and at least 25 of the 30 must be usable."""
    c = 8
    panel, scene, cams, V, target = case(c)
    plan = lfd.Plan(panel, views_per_cluster=c)
    s = lfd.scene_to_device(scene)
    img, _ = plan.render(s, cams)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    grads = {k: v.double().cpu().numpy().reshape(-1) for k, v in plan.backward(s, cams, 2.0 * (img - tgt)).items()}
    plan.close()
    base = {k: torch.tensor(np.asarray(v, np.float64)) for k, v in scene.items()}
    tgt64 = torch.from_numpy(target)

    def loss(params):
        with torch.no_grad():
            return float(((torch_render.render(params, cams, V, c) - tgt64) ** 2).sum())

    def central(key, f, h):
        plus = {k: v.clone() for k, v in base.items()}
        minus = {k: v.clone() for k, v in base.items()}
        plus[key].view(-1)[f] += h
        minus[key].view(-1)[f] -= h
        return (loss(plus) - loss(minus)) / (2 * h)

    used = 0
    for key in KEYS:
        g = grads[key]
        for f in np.argsort(-np.abs(g))[:6]:
            h = 1e-5 * max(1.0, abs(float(base[key].view(-1)[f])))
            d1, d2 = central(key, f, h), central(key, f, 2 * h)
            if abs(d1 - d2) > 1e-3 * max(abs(d1), 1e-12):
                continue  # a threshold lies within 2h: not a smooth point
            used += 1
            assert abs(g[f] - d1) <= 2e-2 * abs(d1) + 1e-4 * float(np.abs(g).max()), (key, int(f), g[f], d1)
    assert used >= 25, used


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
