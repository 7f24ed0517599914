"""Pins of the oracle's subpixel blend (Sec. 4.3, Eq. 9-10, 3DGS rules)."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth

C0 = 0.28209479177387814


def _scene(means, scales, opac, colours):
    m = len(means)
    sh = np.zeros((m, 16, 3), np.float32)
    sh[:, 0, :] = (np.asarray(colours, np.float64) - 0.5) / C0
    return {"means": np.asarray(means, np.float32), "scales": np.asarray(scales, np.float32),
            "quats": np.tile(np.float32([1, 0, 0, 0]), (m, 1)),
            "opacities": np.asarray(opac, np.float32), "sh": sh}


def _cams(baselines, f=200.0, cx=64.5, cy=48.5):
    out = np.zeros((len(baselines), 16), np.float32)
    for j, b in enumerate(baselines):
        out[j, 0:9] = np.eye(3).reshape(-1)
        out[j, 9:12] = (-b, 0.0, 0.0)
        out[j, 12:16] = (f, f, cx, cy)
    return out


def _alpha_closed(o, q):
    v = o * np.exp(-0.5 * q)
    return np.where(v >= 1 / 255, np.minimum(0.99, v), 0.0), v


def test_single_gaussian_closed_form_every_subpixel():
    # One isotropic Gaussian, scale s at depth Z, seen by three cameras that
    # differ by a horizontal baseline, one cluster (reuse): each subpixel sees
    # the mean of its own view (Eq. 5, 10) and the representative view's
    # covariance, here the on-axis one: Sigma2D = ((f s/Z)^2 + 0.3) I.
    f, s, Z, o = 200.0, 0.04, 3.0, 0.85
    base = [-0.05, 0.0, 0.05]
    W, H = 128, 96
    panel = synth.Panel(W, H, 3, 0.2, 3.7, 0.0)
    V = oracle.view_index(panel)
    col = (0.9, 0.4, 0.2)
    scene = _scene([[0.0, 0.0, Z]], [[s, s, s]], [o], [col])
    proj = oracle.project(scene, _cams(base, f), W, H, 3)
    img, _ = oracle.render(proj, V, 3, mode=0)
    sig2 = (f * float(np.float32(s)) / Z) ** 2 + 0.3
    colf = np.array([float(np.float32((c - 0.5) / C0)) * C0 + 0.5 for c in col])
    x = np.arange(W)[None, :, None] + 0.5
    y = np.arange(H)[:, None, None] + 0.5
    mux = f * (0.0 - np.asarray(base, np.float32).astype(np.float64)) / Z + 64.5
    q = ((x - mux[V]) ** 2 + (y - 48.5) ** 2) / sig2
    a, v = _alpha_closed(float(np.float32(o)), q)
    expect = colf[None, None, :] * a
    near = np.abs(v - 1 / 255) < 1e-9
    assert not near.any()
    np.testing.assert_allclose(img, expect, rtol=1e-9, atol=1e-12)
    assert (img > 0).sum() > 300


def test_two_gaussians_closed_form_and_depth_order():
    f, W, H = 200.0, 64, 48
    panel = synth.Panel(W, H, 1, 0.0, 5.0, 0.0)
    V = oracle.view_index(panel)
    c1, c2 = (0.8, 0.1, 0.3), (0.2, 0.7, 0.5)
    cams = _cams([0.0], f, 32.5, 24.5)
    for z1, z2 in ((2.0, 3.0), (3.0, 2.0)):
        scene = _scene([[0.0, 0.0, z1], [0.0, 0.0, z2]], [[0.03] * 3, [0.05] * 3], [0.7, 0.6],
                       [c1, c2])
        proj = oracle.project(scene, cams, W, H, 1)
        img, _ = oracle.render(proj, V, 1, mode=0)
        x = np.arange(W)[None, :] + 0.5
        y = np.arange(H)[:, None] + 0.5
        alphas, cols = [], []
        for i, (mx, z, s) in enumerate(((0.0, z1, 0.03), (0.0, z2, 0.05))):
            sig2 = (f * float(np.float32(s)) / z) ** 2 + 0.3
            mu = f * float(np.float32(mx)) / z + 32.5
            a, _ = _alpha_closed(float(np.float32([0.7, 0.6][i])), ((x - mu) ** 2 + (y - 24.5) ** 2) / sig2)
            alphas.append(a)
            cols.append(proj["color"][0, i])
        front, back = (0, 1) if z1 < z2 else (1, 0)
        expect = (cols[front][None, None, :] * alphas[front][..., None]
                  + cols[back][None, None, :] * (alphas[back] * (1 - alphas[front]))[..., None])
        np.testing.assert_allclose(img, expect, rtol=1e-9, atol=1e-12)


def test_termination_stops_before_adding():
    # Three opaque Gaussians centred on a pixel centre: alpha = 0.99 each. The
    # first two are added (T = 1e-4 after them, not below); the third would
    # take T to 1e-6 < 1e-4, so blending stops without adding it.
    W, H = 16, 16
    panel = synth.Panel(W, H, 1, 0.0, 5.0, 0.0)
    V = oracle.view_index(panel)
    cols = [(0.9, 0.0, 0.0), (0.0, 0.9, 0.0), (0.0, 0.0, 0.9)]
    scene = _scene([[0, 0, 2.0], [0, 0, 3.0], [0, 0, 4.0]], [[0.05] * 3] * 3, [1.0, 1.0, 1.0], cols)
    proj = oracle.project(scene, _cams([0.0], 200.0, 8.5, 8.5), W, H, 1)
    img, _ = oracle.render(proj, V, 1, mode=0)
    c = proj["color"][0]
    a = 0.99
    expect = c[0] * a + c[1] * a * (1 - a)
    np.testing.assert_allclose(img[8, 8], expect, rtol=1e-12)
    # had the third been added, blue would carry c3 * 0.99 * 1e-4
    assert img[8, 8, 2] == 0.0


def _textbook_3dgs(proj, W, H):
    """Vectorised single-view 3DGS: depth-sorted alphas, exclusive cumulative
    transmittance, cut at the first Gaussian that would drop T below 1e-4."""
    valid = proj["valid"][0].astype(bool) & proj["vvalid"][0].astype(bool)
    idx = np.nonzero(valid)[0]
    idx = idx[np.lexsort((idx, proj["depth"][0, idx]))]
    mu = proj["mean2d"][0, idx]
    con = proj["conic"][0, idx]
    col = proj["color"][0, idx]
    o = proj["opac"][idx]
    x = np.arange(W)[None, :, None] + 0.5
    y = np.arange(H)[:, None, None] + 0.5
    dx, dy = x - mu[None, None, :, 0], y - mu[None, None, :, 1]
    q = con[:, 0] * dx * dx + 2 * con[:, 1] * dx * dy + con[:, 2] * dy * dy
    v = o * np.exp(-0.5 * q)
    a = np.where(v >= 1 / 255, np.minimum(0.99, v), 0.0)
    T_after = np.cumprod(1 - a, axis=-1)
    T_before = np.concatenate([np.ones_like(a[..., :1]), T_after[..., :-1]], axis=-1)
    stop = (T_after < 1e-4) & (a > 0)
    first = np.where(stop.any(-1), stop.argmax(-1), a.shape[-1])
    keep = np.arange(a.shape[-1])[None, None, :] < first[..., None]
    w = np.where(keep, a * T_before, 0.0)
    return np.einsum("hwn,nc->hwc", w, col)


def test_one_view_equals_textbook_3dgs():
    # N = 1: every subpixel has view 0 and the render is plain 3DGS.
    W, H = 48, 32
    rng = np.random.default_rng(7)
    m = 120
    means = np.c_[rng.uniform(-0.4, 0.4, (m, 2)), rng.uniform(1.5, 3.0, m)]
    scene = {"means": means.astype(np.float32),
             "scales": np.exp(rng.normal(-3.0, 0.4, (m, 3))).astype(np.float32),
             "quats": rng.normal(size=(m, 4)).astype(np.float32),
             "opacities": (1 / (1 + np.exp(-rng.normal(1.0, 1.5, m)))).astype(np.float32),
             "sh": rng.normal(0, 0.3, (m, 16, 3)).astype(np.float32)}
    proj = oracle.project(scene, _cams([0.0], 60.0, 24.0, 16.0), W, H, 1)
    V = oracle.view_index(synth.Panel(W, H, 1, 0.2, 5.3))
    assert (V == 0).all()
    img, _ = oracle.render(proj, V, 1, mode=0)
    ref = _textbook_3dgs(proj, W, H)
    np.testing.assert_allclose(img, ref, rtol=1e-10, atol=1e-12)
    assert img.max() > 0.5


@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w, 400)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    V = oracle.view_index(w.panel)
    return w, scene, cams, V


def test_one_view_per_cluster_equals_fullframe_then_interlace(tiny):
    # C = 1 (no reuse): the subpixel render equals rendering every view in
    # full and sampling each subpixel from its view's image (Sec. 1, 4.1).
    w, scene, cams, V = tiny
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, 1)
    crop = (40, 30, 200, 110)
    sub, _ = oracle.render(proj, V, 1, crop=crop, mode=0)
    full = oracle.render_fullframe(proj, V, crop=crop)
    np.testing.assert_array_equal(sub, full)
    assert sub.max() > 0.3


@pytest.mark.parametrize("C", [1, 3, 8])
def test_binned_equals_brute_force(tiny, C):
    w, scene, cams, V = tiny
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, C)
    brute, nb = oracle.render(proj, V, C, mode=0)
    binned, nl = oracle.render(proj, V, C, mode=1, tile=(16, 16))
    np.testing.assert_array_equal(brute, binned)
    assert nl < nb


def test_blend_lists_equals_definition(tiny):
    # lists holding every valid Gaussian of the cluster in (depth, id) order
    w, scene, cams, V = tiny
    C = 4
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, C)
    K = proj["conic"].shape[0]
    T = (w.panel.width // 16) * (w.panel.height // 16)
    parts, ranges, pos = [], np.zeros((T, K, 2), np.uint32), 0
    for t in range(T):
        for k in range(K):
            idx = np.nonzero(proj["valid"][k])[0]
            idx = idx[np.lexsort((idx, proj["depth"][k, idx]))]
            ranges[t, k] = (pos, pos + len(idx))
            parts.append(idx)
            pos += len(idx)
    lst = np.concatenate(parts).astype(np.uint32)
    a, _ = oracle.blend_lists(proj, V, C, ranges, lst)
    b, _ = oracle.render(proj, V, C, mode=0)
    np.testing.assert_array_equal(a, b)


def test_background_and_empty_scene():
    W, H = 20, 10
    V = oracle.view_index(synth.Panel(W, H, 2, 0.1, 4.0))
    scene = _scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)))
    proj = oracle.project(scene, _cams([0.0, 0.1]), W, H, 1)
    img, n = oracle.render(proj, V, 1, mode=0, bg=(0.25, 0.5, 1.0))
    assert n == 0
    np.testing.assert_array_equal(img, np.broadcast_to([0.25, 0.5, 1.0], (H, W, 3)))


def test_alpha_threshold_parameter():
    # One Gaussian with peak opacity o: raising the skip threshold above o
    # removes it everywhere; the default threshold is restored afterwards.
    W, H = 16, 16
    V = oracle.view_index(synth.Panel(W, H, 1, 0.0, 5.0, 0.0))
    scene = _scene([[0, 0, 2.0]], [[0.05] * 3], [0.5], [(0.9, 0.9, 0.9)])
    proj = oracle.project(scene, _cams([0.0], 200.0, 8.5, 8.5), W, H, 1)
    base, _ = oracle.render(proj, V, 1, mode=0)
    with oracle.alpha_min(0.51):
        gone, _ = oracle.render(proj, V, 1, mode=0)
    again, _ = oracle.render(proj, V, 1, mode=0)
    assert base.max() > 0.3 and gone.max() == 0.0
    np.testing.assert_array_equal(base, again)
