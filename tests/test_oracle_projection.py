"""Pins of the oracle's FP64 projection (Sec. 3.3, Eq. 4-6)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from paper_2605_04509_gb300 import synth


def _camera(R=np.eye(3), t=np.zeros(3), f=300.0, cx=64.0, cy=48.0):
    c = np.zeros(16, dtype=np.float32)
    c[0:9] = np.asarray(R).reshape(-1)
    c[9:12] = t
    c[12:16] = (f, f, cx, cy)
    return c


def _scene(means, scales, quats, opac, sh):
    return {"means": np.asarray(means, np.float32), "scales": np.asarray(scales, np.float32),
            "quats": np.asarray(quats, np.float32), "opacities": np.asarray(opac, np.float32),
            "sh": np.asarray(sh, np.float32)}


def _conic_to_cov(conic):
    a, b, c = conic
    return np.linalg.inv(np.array([[a, b], [b, c]]))


def test_isotropic_on_axis_closed_form():
    # An isotropic Gaussian of scale s on the optical axis at depth Z projects
    # to the principal point with Sigma2D = ((f s / Z)^2 + 0.3) I, depth Z.
    f, s, Z = 300.0, 0.05, 4.0
    rng = np.random.default_rng(0)
    q = rng.normal(size=(1, 4))
    scene = _scene([[0.0, 0.0, Z]], [[s, s, s]], q, [0.8], np.zeros((1, 16, 3)))
    cams = _camera(f=f)[None]
    p = oracle.project(scene, cams, 128, 96, 1)
    assert p["vvalid"][0, 0] and p["valid"][0, 0]
    np.testing.assert_allclose(p["mean2d"][0, 0], [64.0, 48.0], atol=1e-12)
    cov = _conic_to_cov(p["conic"][0, 0])
    # s, f, Z are float32-exact; the rotation is float32-normalised, hence 1e-6
    sig2 = (f * float(np.float32(s)) / Z) ** 2 + 0.3
    np.testing.assert_allclose(cov, sig2 * np.eye(2), rtol=1e-6, atol=1e-7)
    assert p["depth"][0, 0] == pytest.approx(Z)
    assert p["tau"][0, 0] == pytest.approx(2 * math.log(255 * np.float32(0.8)))


def test_mean_is_inverse_of_backprojection():
    # A point built by back-projecting pixel (u, v) at depth Z from a posed
    # camera must project back to (u, v).
    rig = synth.Rig(5, 40.0, 4.0, 50.0)
    cams = synth.arc_cameras(rig, 128, 96)
    rng = np.random.default_rng(1)
    pts, pix = [], []
    for j in range(5):
        R = cams[j, :9].astype(np.float64).reshape(3, 3)
        t = cams[j, 9:12].astype(np.float64)
        f, _, cx, cy = cams[j, 12:16].astype(np.float64)
        u, v, Z = rng.uniform(0, 128), rng.uniform(0, 96), rng.uniform(2, 6)
        pc = np.array([(u - cx) / f * Z, (v - cy) / f * Z, Z])
        pts.append(R.T @ (pc - t))
        pix.append((j, u, v))
    pts = np.array(pts, dtype=np.float32)
    m = len(pts)
    scene = _scene(pts, np.full((m, 3), 0.05), np.tile([1, 0, 0, 0], (m, 1)), np.full(m, 0.5),
                   np.zeros((m, 16, 3)))
    p = oracle.project(scene, cams, 128, 96, 1)
    for i, (j, u, v) in enumerate(pix):
        # float32 rounding of the point limits agreement to ~1e-4 px
        np.testing.assert_allclose(p["mean2d"][j, i], [u, v], atol=2e-4)


def test_covariance_matches_finite_difference_jacobian():
    # Sigma2D = J W Sigma3D W^T J^T + 0.3 I with J the Jacobian of the pinhole
    # map at the mean (finite differences here) and Sigma3D = R S S^T R^T with
    # R from an independent quaternion->matrix routine.
    rng = np.random.default_rng(2)
    m = 40
    means = rng.uniform(-0.5, 0.5, (m, 3)).astype(np.float32)
    scales = np.exp(rng.normal(-2.5, 0.5, (m, 3))).astype(np.float32)
    quats = rng.normal(size=(m, 4)).astype(np.float32)
    opac = np.full(m, 0.9, np.float32)
    cams = synth.arc_cameras(synth.Rig(3, 30.0, 3.0, 50.0), 160, 120)
    p = oracle.project(_scene(means, scales, quats, opac, np.zeros((m, 16, 3))), cams, 160, 120, 1)
    for j in range(3):
        R = cams[j, :9].astype(np.float64).reshape(3, 3)
        t = cams[j, 9:12].astype(np.float64)
        f, _, cx, cy = cams[j, 12:16].astype(np.float64)

        def proj(pc):
            return np.array([f * pc[0] / pc[2] + cx, f * pc[1] / pc[2] + cy])

        for i in range(m):
            pc = R @ means[i].astype(np.float64) + t
            J = np.zeros((2, 3))
            for a in range(3):
                h = 1e-6 * max(1.0, abs(pc[a]))
                e = np.zeros(3)
                e[a] = h
                J[:, a] = (proj(pc + e) - proj(pc - e)) / (2 * h)
            q = quats[i].astype(np.float64)
            Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
            S3 = Rq @ np.diag(scales[i].astype(np.float64) ** 2) @ Rq.T
            S2 = J @ R @ S3 @ R.T @ J.T + 0.3 * np.eye(2)
            np.testing.assert_allclose(_conic_to_cov(p["conic"][j, i]), S2, rtol=1e-6, atol=1e-9)
            # the depth is kept in FP32 (the precision of the Eq. 11 key)
            assert p["depth"][j, i] == pytest.approx(pc[2], rel=3e-7)


def test_jacobian_clamp_off_screen():
    # 3DGS clamps x/z (and y/z) to 1.3 tan(fov/2) before forming J.
    f, W, H = 100.0, 100, 100
    lim = 1.3 * (0.5 * W / f)
    Z = 2.0
    X = 3.0 * lim * Z  # far right of the frustum
    s = 0.1
    scene = _scene([[X, 0.0, Z]], [[s, s, s]], [[1, 0, 0, 0]], [0.9], np.zeros((1, 16, 3)))
    p = oracle.project(scene, _camera(f=f, cx=50, cy=50)[None], W, H, 1)
    J = np.array([[f / Z, 0, -f * lim / Z], [0, f / Z, 0]])
    S2 = J @ (float(np.float32(s)) ** 2 * np.eye(3)) @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(_conic_to_cov(p["conic"][0, 0]), S2, rtol=1e-9)


def _real_sh(l, m, d):
    th = math.acos(max(-1.0, min(1.0, d[2])))
    ph = math.atan2(d[1], d[0])
    if m < 0:
        return math.sqrt(2) * np.imag(sph_harm_y(l, -m, th, ph))
    if m == 0:
        return np.real(sph_harm_y(l, 0, th, ph))
    return math.sqrt(2) * np.real(sph_harm_y(l, m, th, ph))


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_sh_colour_matches_legendre_real_sh(degree):
    # colour = max(0, sum_lm Y_lm(dir) h_lm + 0.5), Y_lm the real SH built
    # from scipy's associated-Legendre spherical harmonics (Condon-Shortley
    # phase, sqrt(2) Re/Im for m != 0), dir from the camera centre to the mean.
    rng = np.random.default_rng(3 + degree)
    m = 25
    dirs = rng.normal(size=(m, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dirs[:, 2] = np.abs(dirs[:, 2]) + 0.3  # in front of the camera
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    means = (dirs * 3.0).astype(np.float32)
    sh = rng.normal(0, 0.3, (m, 16, 3)).astype(np.float32)
    scene = _scene(means, np.full((m, 3), 0.05), np.tile([1, 0, 0, 0], (m, 1)), np.full(m, 0.5), sh)
    p = oracle.project(scene, _camera()[None], 128, 96, 1, sh_degree=degree)
    for i in range(m):
        d = means[i].astype(np.float64)
        d /= np.linalg.norm(d)
        basis = [_real_sh(l, mm, d) for l in range(degree + 1) for mm in range(-l, l + 1)]
        expect = np.maximum(np.array(basis) @ sh[i, : len(basis)].astype(np.float64) + 0.5, 0.0)
        np.testing.assert_allclose(p["color"][0, i], expect, rtol=1e-9, atol=1e-12)


def test_dc_only_colour_closed_form():
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 0] = [0.5, -3.0, 1.0]
    scene = _scene([[0.1, 0.2, 3.0]], [[0.05] * 3], [[1, 0, 0, 0]], [0.5], sh)
    p = oracle.project(scene, _camera()[None], 128, 96, 1)
    c0 = 0.28209479177387814
    np.testing.assert_allclose(p["color"][0, 0], [c0 * 0.5 + 0.5, 0.0, c0 + 0.5], rtol=1e-12)


def test_culling_near_plane_and_low_opacity():
    scene = _scene([[0, 0, 0.1], [0, 0, 3.0], [0, 0, 3.0]], [[0.05] * 3] * 3,
                   [[1, 0, 0, 0]] * 3, [0.9, 1.0 / 256.0, 0.9], np.zeros((3, 16, 3)))
    p = oracle.project(scene, _camera()[None], 128, 96, 1)
    assert p["vvalid"][0].tolist() == [0, 1, 1]
    assert p["valid"][0].tolist() == [0, 0, 1]
    # at q = tau the opacity o exp(-q/2) sits exactly on the 1/255 threshold
    assert 0.9 * math.exp(-p["tau"][0, 2] / 2) == pytest.approx(1 / 255, rel=1e-6)


def test_cluster_attributes_come_from_representative():
    # Eq. 6: with clusters of C views, cluster k carries the covariance, depth
    # and colour of its representative view; per-view means stay per view.
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w, 300)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    p1 = oracle.project(scene, cams, w.panel.width, w.panel.height, 1)
    for C in (2, 3, 8):
        pc = oracle.project(scene, cams, w.panel.width, w.panel.height, C)
        _slot, rep = oracle.clusters(8, C)
        np.testing.assert_array_equal(pc["mean2d"], p1["mean2d"])
        for k, r in enumerate(rep):
            for key in ("conic", "depth", "color", "tau", "valid"):
                np.testing.assert_array_equal(pc[key][k], p1[key][r])
