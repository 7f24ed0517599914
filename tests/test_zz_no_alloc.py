"""lfd_render_projected_noalloc against lfd_render_projected.

The allocation-free entry point serves callers that must not allocate device
memory while they render (a real-time loop that cannot afford the
synchronisation an allocation implies, or a host whose own memory manager owns
the device heap). Its scratch lives in one fixed device array inside the
library, so it handles small frames only. This file runs last so that a
failure here does not hide any other test's result.
"""
import numpy as np
import pytest

from paper_2605_04509_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402


@pytest.mark.parametrize("c,sort_mode,spt", [(8, lfd.SORT_DEPTH_FIRST, 0), (1, lfd.SORT_DEPTH_FIRST, 0),
                                             (4, lfd.SORT_KEY64, 0), (8, lfd.SORT_DEPTH_FIRST, 2)])
def test_noalloc_matches_allocating_entry_point(c, sort_mode, spt):
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    # spt: the plan's subpixels-per-thread option reaches the blend of both calls
    plan = lfd.Plan(w.panel, views_per_cluster=c, sort_mode=sort_mode, bg=(0.05, 0.1, 0.2),
                    subpixels_per_thread=spt)
    attrs = plan.project(lfd.scene_to_device(scene), cams)
    want, st = plan.render_projected(attrs)
    want = want.clone()
    assert st["num_pairs"] > 1000
    # two calls in a row: the shared scratch keeps the first call's contents
    for _ in range(2):
        got, st2 = plan.render_projected_noalloc(attrs)
        torch.cuda.synchronize()
        assert st2["num_pairs"] == st["num_pairs"]
        # same kernels, same order of operations: identical bits
        assert torch.equal(got, want)
    plan.close()


def test_noalloc_rejects_frames_beyond_its_limits():
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w, 40000)  # 40,000 Gaussians x 1 cluster > 32,768 items
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    attrs = plan.project(lfd.scene_to_device(scene), cams)
    with pytest.raises(lfd.LFDError) as e:
        plan.render_projected_noalloc(attrs)
    assert e.value.status == lfd.LFD_ERR_CAPACITY
    plan.close()
