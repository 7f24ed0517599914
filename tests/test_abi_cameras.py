"""lfd_make_arc_cameras (the view-cone input of the problem statement, reading
D-l of the camera placement) against the seeded input generator's cameras, on
the rigs of all five workloads, and its argument checks. Host only: no GPU."""
import ctypes
import math

import numpy as np
import pytest

from paper_2605_04509_gb300 import synth

RIGS = [
    ("tiny", synth.WORKLOADS["tiny"].rig, 256, 144),
    ("paper4k", synth.WORKLOADS["paper4k"].rig, 3840, 2160),
    ("precision8k", synth.WORKLOADS["precision8k"].rig, 7680, 4320),
    ("diff1080", synth.WORKLOADS["diff1080"].rig, 1920, 1080),
    ("batching 1536x2048/48", synth.Rig(48, 35.0, 30.0, 50.0), 1536, 2048),
    ("one view", synth.Rig(1, 40.0, 30.0, 50.0), 640, 480),
]


@pytest.fixture(scope="module")
def lfd():
    from paper_2605_04509_gb300 import build_lib, lfd as mod
    build_lib.build()
    mod.load()
    return mod


@pytest.mark.parametrize("name,rig,w,h", RIGS, ids=[r[0] for r in RIGS])
def test_arc_cameras_match_generator(lfd, name, rig, w, h):
    got = lfd.make_arc_cameras(rig.num_views, rig.cone_deg, rig.radius, rig.fov_x_deg, w, h)
    want = synth.arc_cameras(rig, w, h)
    assert got.shape == want.shape == (rig.num_views, 16)
    # both evaluate in double and round to float: equal up to one float ulp
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=2e-7 * max(1.0, rig.radius))


def test_arc_cameras_geometry(lfd):
    # independent checks: rotations orthonormal, centres on the arc, the
    # origin projects to the principal point, view 0 on the left (x < 0)
    rig = synth.WORKLOADS["paper4k"].rig
    cams = lfd.make_arc_cameras(rig.num_views, rig.cone_deg, rig.radius, rig.fov_x_deg, 3840, 2160)
    for j, c in enumerate(cams.astype(np.float64)):
        R = c[:9].reshape(3, 3)
        t = c[9:12]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-6)
        centre = -R.T @ t
        assert np.linalg.norm(centre) == pytest.approx(rig.radius, rel=1e-6)
        th = math.radians(-rig.cone_deg / 2 + rig.cone_deg * j / (rig.num_views - 1))
        np.testing.assert_allclose(centre, [rig.radius * math.sin(th), 0.0, -rig.radius * math.cos(th)],
                                   atol=1e-5)
        o = R @ np.zeros(3) + t  # the world origin in camera space
        assert o[2] == pytest.approx(rig.radius, rel=1e-6)
        assert c[12] * o[0] / o[2] + c[14] == pytest.approx(1920.0, abs=1e-3)
        assert c[13] * o[1] / o[2] + c[15] == pytest.approx(1080.0, abs=1e-3)
    assert c[12] == pytest.approx(1920.0 / math.tan(math.radians(25.0)), rel=1e-6)
    assert (-cams[0, :9].reshape(3, 3).T @ cams[0, 9:12])[0] < 0


def test_arc_cameras_argument_checks(lfd):
    L = lfd.load()
    buf = (lfd.CCamera * 4)()
    assert L.lfd_make_arc_cameras(4, 40.0, 30.0, 50.0, 64, 64, None) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(0, 40.0, 30.0, 50.0, 64, 64, buf) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(256, 40.0, 30.0, 50.0, 64, 64, buf) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(4, 40.0, 0.0, 50.0, 64, 64, buf) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(4, 40.0, 30.0, 180.0, 64, 64, buf) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(4, 40.0, 30.0, 50.0, 0, 64, buf) == lfd.LFD_ERR_INVALID
    assert L.lfd_make_arc_cameras(4, 40.0, 30.0, 50.0, 64, 64, buf) == lfd.LFD_OK
    assert isinstance(ctypes.sizeof(buf), int)
