"""Pins of the differentiable FP64 oracle (oracle/torch_render.py), the
reference gradient of the backward pass: its forward equals the C oracle's,
and its autograd gradient equals central finite differences."""
import numpy as np
import pytest
import torch

import oracle
from oracle import torch_render
from paper_2605_04509_gb300 import synth


def small_case(m=150, seed=3, n_views=4, c=2):
    panel = synth.Panel(64, 48, n_views, 0.2, 4.3, 0.0)
    rig = synth.Rig(n_views, 20.0, 4.0, 50.0)
    scene = synth.uniform_scene(m, seed)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    V = oracle.view_index(panel)
    return panel, scene, cams, V, c


def to_params(scene, requires_grad=True):
    return {k: torch.tensor(np.asarray(v, np.float64), requires_grad=requires_grad)
            for k, v in scene.items()}


@pytest.mark.parametrize("c", [1, 2, 4])
def test_forward_equals_c_oracle(c):
    panel, scene, cams, V, _ = small_case(c=c)
    img = torch_render.render(to_params(scene, False), cams, V, c, bg=(0.1, 0.2, 0.3)).numpy()
    proj = oracle.project(scene, cams, panel.width, panel.height, c)
    ref, _ = oracle.render(proj, V, c, mode=0, bg=(0.1, 0.2, 0.3))
    np.testing.assert_allclose(img, ref, rtol=1e-10, atol=1e-12)
    assert img.max() > 0.3


@pytest.mark.parametrize("rel", [-1e-3, 1e-3, 0.5])
def test_forward_with_moved_threshold_equals_c_oracle(rel):
    # the skip threshold moved as the bracket of the accuracy reading does
    # (and far, to see that it acts): same image as the C oracle's
    panel, scene, cams, V, _ = small_case(c=2)
    a = oracle.ALPHA_MIN * (1 + rel)
    img = torch_render.render(to_params(scene, False), cams, V, 2, alpha_min=a).numpy()
    proj = oracle.project(scene, cams, panel.width, panel.height, 2)
    with oracle.alpha_min(a):
        ref, _ = oracle.render(proj, V, 2, mode=0)
    np.testing.assert_allclose(img, ref, rtol=1e-10, atol=1e-12)
    if rel == 0.5:
        base = torch_render.render(to_params(scene, False), cams, V, 2).numpy()
        assert np.abs(base - img).max() > 1e-3


def _loss(params, cams, V, c, target):
    img = torch_render.render(params, cams, V, c)
    return ((img - target) ** 2).sum()


def test_autograd_matches_central_differences():
    panel, scene, cams, V, c = small_case(m=60, seed=11)
    rng = np.random.default_rng(4)
    target = torch.tensor(rng.uniform(0, 1, (panel.height, panel.width, 3)))
    params = to_params(scene)
    loss = _loss(params, cams, V, c, target)
    loss.backward()
    checked = 0
    for key in ("means", "scales", "quats", "opacities", "sh"):
        g = params[key].grad.numpy()
        flat = np.argsort(-np.abs(g).reshape(-1))[:6]  # the most influential entries
        for f in flat:
            base = {k: v.detach().clone() for k, v in params.items()}
            h = 1e-6 * max(1.0, abs(float(base[key].reshape(-1)[f])))
            plus = {k: v.clone() for k, v in base.items()}
            minus = {k: v.clone() for k, v in base.items()}
            plus[key].view(-1)[f] += h
            minus[key].view(-1)[f] -= h
            with torch.no_grad():
                fd = (_loss(plus, cams, V, c, target) - _loss(minus, cams, V, c, target)) / (2 * h)
            an = g.reshape(-1)[f]
            assert abs(fd.item() - an) <= 1e-4 * max(1.0, abs(an)), (key, f, fd.item(), an)
            checked += 1
    assert checked == 30
