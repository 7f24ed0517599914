"""Capacity mode (frames without host read-back), CUDA-graph capture and
batched multi-scene rendering, against the single-scene entry point.

The image of a frame does not depend on how it was scheduled: capacity-mode
frames, graph replays and every scene of a batch must equal lfd_render of
the same scene bit for bit (the single-scene path itself is held to the
oracle by test_gpu_parity.py). Overflow must leave the images untouched and
be reported; a bounded device wait must give up and report.
"""
import numpy as np
import pytest

from paper_2605_04509_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402

PANEL_B = synth.Panel(200, 120, 13, 0.2027, 5.3, 0.7)
RIG_B = synth.Rig(13, 30.0, 4.0, 50.0)


def scene_case(panel, rig, m, seed):
    scene = synth.uniform_scene(m, seed)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    return scene, cams


def reference(plan, scene_dev, cams):
    img, st = plan.render(scene_dev, cams)
    torch.cuda.synchronize()
    return img.clone(), st["num_pairs"]


@pytest.mark.parametrize("c", [8, 1])
def test_capacity_mode_equals_plain_frame(c):
    w = synth.WORKLOADS["tiny"]
    scene = lfd.scene_to_device(synth.scene_for(w))
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    plan = lfd.Plan(w.panel, views_per_cluster=c, bg=(0.1, 0.0, 0.3))
    want, P = reference(plan, scene, cams)
    plan.reserve(scene["means"].shape[0], P + 1000)
    for _ in range(2):
        got, st = plan.render(scene, cams)
        assert st["num_pairs"] == -1
        assert plan.status() == P
        assert torch.equal(got, want)
    plan.close()


def test_capacity_overflow_leaves_image_and_reports():
    w = synth.WORKLOADS["tiny"]
    scene = lfd.scene_to_device(synth.scene_for(w))
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    want, P = reference(plan, scene, cams)
    plan.reserve(scene["means"].shape[0], P - 1)
    out = torch.full_like(want, -7.0)
    plan.render(scene, cams, out=out)
    rc, P_seen = plan.status_code()
    assert rc == lfd.LFD_ERR_CAPACITY and P_seen == P
    assert torch.all(out == -7.0)
    assert plan.status_code()[0] == lfd.LFD_OK  # the flag was cleared
    plan.reserve(scene["means"].shape[0], P)
    plan.render(scene, cams, out=out)
    assert plan.status() == P
    assert torch.equal(out, want)
    # more Gaussians than reserved: refused on the host
    big = lfd.scene_to_device(synth.scene_for(w, 3000))
    with pytest.raises(lfd.LFDError) as e:
        plan.render(big, cams)
    assert e.value.status == lfd.LFD_ERR_CAPACITY
    plan.close()


def test_graph_capture_and_replay():
    w = synth.WORKLOADS["tiny"]
    host = synth.scene_for(w)
    scene = lfd.scene_to_device(host)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    plan = lfd.Plan(w.panel, views_per_cluster=4)
    want, P = reference(plan, scene, cams)
    plan.reserve(scene["means"].shape[0], 2 * P)
    out = torch.zeros_like(want)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.render(scene, cams, out=out)  # uncaptured frame: attributes, warm-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    launches0 = lfd.kernel_launches()
    with torch.cuda.graph(graph, stream=s):
        plan.render(scene, cams, out=out)
    assert lfd.kernel_launches() > launches0
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert plan.status() == P
    assert torch.equal(out, want)
    # new Gaussian values in the captured buffers are rendered by a replay
    moved = dict(host)
    moved["opacities"] = (host["opacities"] * 0.5).astype(np.float32)
    moved_dev = lfd.scene_to_device(moved)
    scene["opacities"].copy_(moved_dev["opacities"])
    graph.replay()
    torch.cuda.synchronize()
    plan.status()
    plan2 = lfd.Plan(w.panel, views_per_cluster=4)
    want2, _ = reference(plan2, moved_dev, cams)
    assert torch.equal(out, want2)
    plan.close()
    plan2.close()


def batch_case():
    w = synth.WORKLOADS["tiny"]
    plan_a = lfd.Plan(w.panel, views_per_cluster=8)
    plan_b = lfd.Plan(PANEL_B, views_per_cluster=4, bg=(0.2, 0.1, 0.0))
    cams_a = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    cams_b = synth.arc_cameras(RIG_B, PANEL_B.width, PANEL_B.height)
    plans = [plan_a, plan_b, plan_a]
    hosts = [synth.uniform_scene(1500, 100), synth.uniform_scene(2500, 101),
             synth.uniform_scene(700, 102)]
    scenes = [lfd.scene_to_device(h) for h in hosts]
    cams = [cams_a, cams_b, cams_a]
    refs, Ps = [], []
    for p, sc, cm in zip(plans, scenes, cams):
        img, P = reference(p, sc, cm)
        refs.append(img)
        Ps.append(P)
    return plans, scenes, cams, refs, Ps


def test_batch_equals_single_scene_frames():
    plans, scenes, cams, refs, Ps = batch_case()
    batch = lfd.Batch(plans)
    batch.reserve([sc["means"].shape[0] for sc in scenes], sum(Ps) + 10)
    for _ in range(2):
        outs = batch.render(scenes, cams)
        assert batch.status() == sum(Ps)
        for got, want in zip(outs, refs):
            assert torch.equal(got, want)
    batch.close()


def test_batch_overflow_and_graph_replay():
    plans, scenes, cams, refs, Ps = batch_case()
    batch = lfd.Batch(plans)
    batch.reserve([sc["means"].shape[0] for sc in scenes], sum(Ps) - 1)
    outs = [torch.full_like(r, 3.0) for r in refs]
    batch.render(scenes, cams, outs=outs)
    rc, P = batch.status_code()
    assert rc == lfd.LFD_ERR_CAPACITY and P == sum(Ps)
    assert all(torch.all(o == 3.0) for o in outs)
    batch.reserve([sc["means"].shape[0] for sc in scenes], sum(Ps))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.render(scenes, cams, outs=outs)
    torch.cuda.synchronize()
    batch.status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.render(scenes, cams, outs=outs)
    for o in outs:
        o.zero_()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == sum(Ps)
    for got, want in zip(outs, refs):
        assert torch.equal(got, want)
    batch.close()


def test_batch_rejects_mixed_plans():
    w = synth.WORKLOADS["tiny"]
    a = lfd.Plan(w.panel, views_per_cluster=8)
    b = lfd.Plan(w.panel, views_per_cluster=8, sort_mode=lfd.SORT_KEY64)
    with pytest.raises(lfd.LFDError) as e:
        lfd.Batch([a, b])
    assert e.value.status == lfd.LFD_ERR_INVALID
    with pytest.raises(lfd.LFDError):
        lfd.Batch([])


@pytest.mark.parametrize("spt", [1, 2, 4, 8])
def test_staging_depth_does_not_change_the_image(spt):
    w = synth.WORKLOADS["tiny"]
    scene = lfd.scene_to_device(synth.scene_for(w))
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    # two views per cluster: runs short enough for one subpixel per thread
    want, _ = reference(lfd.Plan(w.panel, views_per_cluster=2), scene, cams)
    got, _ = reference(lfd.Plan(w.panel, views_per_cluster=2, subpixels_per_thread=spt), scene, cams)
    assert torch.equal(got, want)


def test_bounded_wait_gives_up_and_reports():
    rc = lfd.load().lfd_selftest_wait_timeout(torch.cuda.current_stream().cuda_stream)
    assert rc == lfd.LFD_ERR_TIMEOUT
    # the context is still usable
    x = torch.ones(10, device="cuda")
    assert float(x.sum()) == 10.0


def test_batch_with_an_empty_scene_and_one_scene_batches():
    plans, scenes, cams, refs, Ps = batch_case()
    # a scene without Gaussians renders the background only
    host0 = synth.uniform_scene(1, 103)
    host0 = {k: v[:0] for k, v in host0.items()}
    empty = lfd.scene_to_device(host0)
    batch = lfd.Batch([plans[0], plans[1]])
    batch.reserve([0, scenes[1]["means"].shape[0]], Ps[1] + 10)
    outs = batch.render([empty, scenes[1]], [cams[0], cams[1]])
    assert batch.status() == Ps[1]
    assert torch.equal(outs[1], refs[1])
    assert torch.all(outs[0] == 0.0)  # plan 0 has a black background
    batch.close()
    # a batch of one scene equals the single-scene frame
    one = lfd.Batch([plans[1]])
    one.reserve([scenes[1]["means"].shape[0]], Ps[1])
    out = one.render([scenes[1]], [cams[1]])
    assert one.status() == Ps[1]
    assert torch.equal(out[0], refs[1])
    one.close()


def test_capacity_mode_with_no_gaussians():
    w = synth.WORKLOADS["tiny"]
    host = {k: v[:0] for k, v in synth.scene_for(w).items()}
    scene = lfd.scene_to_device(host)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    plan = lfd.Plan(w.panel, views_per_cluster=8, bg=(0.25, 0.5, 0.75))
    plan.reserve(10, 100)
    out, _ = plan.render(scene, cams)
    assert plan.status() == 0
    img = out.cpu().numpy()
    assert np.all(img[..., 0] == np.float32(0.25)) and np.all(img[..., 2] == np.float32(0.75))
    plan.close()


def test_frames_in_flight_on_two_plans_and_streams():
    # the serving schedule of the benchmark: two capacity-mode plans render
    # alternate frames on their own streams, device-resident and from pinned
    # host buffers; every image equals the single-scene frame
    w = synth.WORKLOADS["tiny"]
    host = synth.scene_for(w)
    scene = lfd.scene_to_device(host)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    ref_plan = lfd.Plan(w.panel, views_per_cluster=8)
    want, P = reference(ref_plan, scene, cams)
    plans = [lfd.Plan(w.panel, views_per_cluster=8) for _ in range(2)]
    for p in plans:
        p.reserve(scene["means"].shape[0], P + 64)
    streams = [torch.cuda.Stream() for _ in range(2)]
    outs = [torch.full_like(want, -1.0) for _ in range(2)]
    for i in range(6):
        plans[i % 2].render(scene, cams, outs[i % 2], streams[i % 2])
    torch.cuda.synchronize()
    for p, o in zip(plans, outs):
        assert p.status() == P
        assert torch.equal(o, want)
    hscene = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
    houts = [torch.full((w.panel.height, w.panel.width, 3), -1.0).pin_memory() for _ in range(2)]
    for i in range(6):
        plans[i % 2].render_host_async(hscene, cams, houts[i % 2], streams[i % 2])
    for p in plans:
        p.render_host_wait()
        assert p.status() == P
    for h in houts:
        assert torch.equal(h, want.cpu())
    for p in plans + [ref_plan]:
        p.close()
