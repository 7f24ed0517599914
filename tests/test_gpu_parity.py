"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bit-exact: view index V, remap table Psi and its cluster runs, tile bins,
Eq. 11 keys, the sorted list and the range table. Tolerance (clamped [0, 1]
images): max |err| <= 2e-3 and at most 0.1 % of subpixels off by more than
1/255, against the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth

from .helpers import assert_image_close, assert_render_matches, image_metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402


def f32_attrs(proj, c):
    """Oracle FP64 projection rounded to the float32 stage layouts."""
    means = oracle.means_by_slot(proj["mean2d"], proj["vvalid"], c).astype(np.float32)
    K, M = proj["depth"].shape
    co = np.zeros((K, M, 4), np.float32)
    co[..., :3] = proj["conic"]
    co[..., 3] = proj["opac"][None, :]
    ct_ = np.zeros((K, M, 4), np.float32)
    ct_[..., :3] = proj["color"]
    ct_[..., 3] = np.where(proj["valid"].astype(bool), proj["tau"], -1.0)
    return {"means2d": np.ascontiguousarray(means), "conic_opacity": co, "color_tau": ct_,
            "depth": proj["depth"].astype(np.float32)}


def to_dev(attrs):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in attrs.items()}


def oracle_proj_from_f32(attrs, num_views, c):
    """The float32 stage inputs as an FP64 oracle projection dict."""
    mean2d, vvalid = oracle.per_view_from_slots(attrs["means2d"].astype(np.float64), num_views, c)
    tau = attrs["color_tau"][..., 3].astype(np.float64)
    return {"mean2d": mean2d, "vvalid": vvalid,
            "conic": np.ascontiguousarray(attrs["conic_opacity"][..., :3], dtype=np.float64),
            "color": np.ascontiguousarray(attrs["color_tau"][..., :3], dtype=np.float64),
            "opac": np.ascontiguousarray(attrs["conic_opacity"][0, :, 3], dtype=np.float64),
            "depth": attrs["depth"].astype(np.float64),
            "valid": (tau >= 0).astype(np.uint8)}


@pytest.fixture(scope="module")
def tiny():
    w = synth.WORKLOADS["tiny"]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    return w, scene, cams


PANELS = [
    synth.WORKLOADS["tiny"].panel,
    synth.Panel(250, 141, 13, 0.2027, 5.3, 0.7),
    synth.Panel(64, 40, 1, 0.0, 4.0, 0.0),
    synth.Panel(97, 33, 255, -0.31, 7.7, -2.5),
]


@pytest.mark.parametrize("panel", PANELS)
@pytest.mark.parametrize("tile,c", [((16, 16), 8), ((8, 8), 1), ((32, 16), 3)])
def test_panel_tables_bit_exact(panel, tile, c):
    plan = lfd.Plan(panel, tile=tile, views_per_cluster=c)
    V, psi, n_sub, seg = plan.tables()
    Vo = oracle.view_index(panel)
    np.testing.assert_array_equal(V, Vo)
    po, no, so = oracle.remap(Vo, panel.num_views, tile[0], tile[1], c)
    np.testing.assert_array_equal(n_sub, no)
    np.testing.assert_array_equal(seg, so)
    for t in range(len(n_sub)):
        np.testing.assert_array_equal(psi[t, : n_sub[t]], po[t, : no[t]])
    plan.close()


def test_panel_tables_paper_4k():
    panel = synth.WORKLOADS["paper4k"].panel
    plan = lfd.Plan(panel, tile=(16, 16), views_per_cluster=8)
    V, psi, n_sub, seg = plan.tables()
    Vo = oracle.view_index(panel)
    np.testing.assert_array_equal(V, Vo)
    po, no, so = oracle.remap(Vo, panel.num_views, 16, 16, 8)
    np.testing.assert_array_equal(seg, so)
    np.testing.assert_array_equal(psi, np.where(np.arange(psi.shape[1])[None] < no[:, None], po, psi))
    plan.close()


@pytest.mark.parametrize("c", [1, 3, 8])
def test_projection_matches_fp64(tiny, c):
    w, scene, cams = tiny
    plan = lfd.Plan(w.panel, views_per_cluster=c)
    out = plan.project(lfd.scene_to_device(scene), cams)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, c)
    ref = f32_attrs(proj, c)
    gm, rm = got["means2d"], ref["means2d"]
    assert np.array_equal(np.isnan(gm), np.isnan(rm))
    fin = np.isfinite(rm)
    np.testing.assert_allclose(gm[fin], rm[fin], rtol=0, atol=2e-3)
    valid = ref["color_tau"][..., 3] >= 0
    assert np.array_equal(got["color_tau"][..., 3] >= 0, valid)
    gc, rc = got["conic_opacity"][valid][:, :3], ref["conic_opacity"][valid][:, :3]
    scale = np.abs(rc).max(axis=1, keepdims=True)
    assert (np.abs(gc - rc) <= 1e-4 * scale + 1e-7).all()
    # the depth (sort-key precision, Eq. 11) is one fixed FP32 sequence on both sides
    np.testing.assert_array_equal(got["depth"][valid], ref["depth"][valid])
    np.testing.assert_allclose(got["color_tau"][valid][:, :3], ref["color_tau"][valid][:, :3],
                               atol=2e-5)
    np.testing.assert_allclose(got["color_tau"][valid][:, 3], ref["color_tau"][valid][:, 3],
                               atol=2e-5)
    plan.close()


@pytest.mark.parametrize("degree", [0, 1, 2])
def test_projection_lower_sh_degrees(tiny, degree):
    # records of fewer than 16 coefficients take the element-wise staging path
    w, scene, cams = tiny
    ncoef = (degree + 1) ** 2
    low = dict(scene)
    low["sh"] = np.ascontiguousarray(scene["sh"][:, :ncoef, :])
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    out = plan.project(lfd.scene_to_device(low), cams)
    torch.cuda.synchronize()
    got = out["color_tau"].cpu().numpy()
    ref = f32_attrs(oracle.project(low, cams, w.panel.width, w.panel.height, 8, sh_degree=degree), 8)
    valid = ref["color_tau"][..., 3] >= 0
    assert valid.sum() > 1000
    assert np.array_equal(got[..., 3] >= 0, valid)
    np.testing.assert_allclose(got[valid][:, :3], ref["color_tau"][valid][:, :3], atol=2e-5)
    plan.close()


def _stage_inputs(w, scene, cams, c):
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, c)
    return f32_attrs(proj, c)


ALL_SORT_MODES = [lfd.SORT_DEPTH_FIRST, lfd.SORT_KEY64]


@pytest.mark.parametrize("sort_mode", ALL_SORT_MODES)
@pytest.mark.parametrize("tile,c", [((16, 16), 8), ((8, 8), 1), ((32, 16), 3), ((16, 8), 5)])
def test_bins_sort_ranges_bit_exact(tiny, sort_mode, tile, c):
    w, scene, cams = tiny
    attrs = _stage_inputs(w, scene, cams, c)
    plan = lfd.Plan(w.panel, tile=tile, views_per_cluster=c, sort_mode=sort_mode)
    _img, st = plan.render_projected(to_dev(attrs))
    ref = oracle.mirror_lists(w.panel.width, w.panel.height, tile,
                              attrs["conic_opacity"][..., :3], attrs["color_tau"][..., 3],
                              attrs["depth"], attrs["means2d"])
    assert st["num_pairs"] == len(ref["list"]) > 1000
    lst, ranges, keys = plan.lists(st["num_pairs"], with_keys=sort_mode == lfd.SORT_KEY64)
    np.testing.assert_array_equal(ranges, ref["ranges"])
    np.testing.assert_array_equal(lst, ref["list"])
    if keys is not None:
        np.testing.assert_array_equal(keys, ref["keys_sorted"])
    plan.close()


# (width, height, tile, largest sigma, Gaussians per cluster): the second panel
# has more than 64 tile columns and 15 tile rows, so the largest ellipses
# overflow the count pass's union descriptor (their units come from the
# geometry) and span several 64-column windows
@pytest.mark.parametrize("width,height,tile,smax,m", [(200, 120, (16, 16), 30.0, 3000),
                                                      (1100, 330, (8, 8), 160.0, 1500)])
def test_bins_random_conics_bit_exact(width, height, tile, smax, m):
    # synthetic ellipses of every orientation and size, many off-panel
    panel = synth.Panel(width, height, 12, 0.15, 5.0, 0.0)
    K, M, C = 3, m, 4
    rng = np.random.default_rng(31)
    conic = synth.random_conics(K * M, 32, 0.6, smax).reshape(K, M, 3)
    tau = rng.uniform(0, 11.0, (K, M)).astype(np.float32)
    tau[rng.uniform(size=(K, M)) < 0.1] = -1.0
    depth = rng.uniform(0.3, 40.0, (K, M)).astype(np.float32)
    base = np.stack([rng.uniform(-40, width + 40, (K, M)), rng.uniform(-40, height + 40, (K, M))], -1)
    means = (base[:, :, None, :] + rng.normal(0, 10.0, (K, M, C, 2))).astype(np.float32)
    means[rng.uniform(size=(K, M, C)) < 0.05] = np.nan
    co = np.concatenate([conic, np.full((K, M, 1), 0.5, np.float32)], -1)
    ct_ = np.concatenate([np.full((K, M, 3), 0.5, np.float32), tau[..., None]], -1)
    attrs = {"means2d": means, "conic_opacity": co, "color_tau": ct_, "depth": depth}
    ref = oracle.mirror_lists(panel.width, panel.height, tile, conic, tau, depth, means)
    if width > 1000:
        # the case reaches the overflow path: unions wider than 64 tile columns
        counts = np.asarray(ref["counts"]).reshape(K, M)
        assert (counts > 15 * 64).sum() > 10
    for sort_mode in ALL_SORT_MODES:
        plan = lfd.Plan(panel, tile=tile, views_per_cluster=C, sort_mode=sort_mode)
        _img, st = plan.render_projected(to_dev(attrs))
        lst, ranges, keys = plan.lists(st["num_pairs"], with_keys=sort_mode == lfd.SORT_KEY64)
        assert st["num_pairs"] == len(ref["list"])
        np.testing.assert_array_equal(lst, ref["list"])
        np.testing.assert_array_equal(ranges, ref["ranges"])
        if keys is not None:
            np.testing.assert_array_equal(keys, ref["keys_sorted"])
        plan.close()


@pytest.mark.parametrize("c", [1, 4, 8])
def test_blend_matches_oracle_on_same_lists(tiny, c):
    w, scene, cams = tiny
    attrs = _stage_inputs(w, scene, cams, c)
    plan = lfd.Plan(w.panel, views_per_cluster=c)
    plan.set_flags(lfd.FLAG_COUNT_EVALS)
    img, st = plan.render_projected(to_dev(attrs))
    ref = oracle.mirror_lists(w.panel.width, w.panel.height, (16, 16),
                              attrs["conic_opacity"][..., :3], attrs["color_tau"][..., 3],
                              attrs["depth"], attrs["means2d"])
    p64 = oracle_proj_from_f32(attrs, w.panel.num_views, c)
    V = oracle.view_index(w.panel)
    want, n_eval = oracle.blend_lists(p64, V, c, ref["ranges"], ref["list"])
    with oracle.alpha_min(oracle.ALPHA_MIN * (1 - 1e-3)):
        lo, _ = oracle.blend_lists(p64, V, c, ref["ranges"], ref["list"])
    with oracle.alpha_min(oracle.ALPHA_MIN * (1 + 1e-3)):
        hi, _ = oracle.blend_lists(p64, V, c, ref["ranges"], ref["list"])
    m = assert_render_matches(img.cpu().numpy(), want, lo, hi, f"blend C={c}")
    assert m["psnr"] > 60
    # the GPU's count of visited list entries agrees with the oracle's walk;
    # the per-view footprint test evaluates only a subset of them
    assert abs(st["num_visits"] - n_eval) <= 1e-3 * n_eval
    assert 0 < st["num_evals"] <= st["num_visits"]
    plan.close()


@pytest.mark.parametrize("c", [1, 3, 8])
@pytest.mark.parametrize("sort_mode", ALL_SORT_MODES)
def test_render_matches_fp64_oracle(tiny, c, sort_mode):
    w, scene, cams = tiny
    plan = lfd.Plan(w.panel, views_per_cluster=c, sort_mode=sort_mode)
    img, st = plan.render(lfd.scene_to_device(scene), cams)
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, c)
    V = oracle.view_index(w.panel)
    ref, lo, hi = oracle.render_bracket(proj, V, c, mode=1)
    m = assert_render_matches(img.cpu().numpy(), ref, lo, hi, f"render C={c}")
    assert m["psnr"] > 60 and st["num_pairs"] > 0
    plan.close()


@pytest.mark.parametrize("tile", [(8, 8), (32, 16), (16, 8)])
def test_render_ragged_panel(tile):
    panel = synth.Panel(250, 141, 13, 0.2027, 5.3, 0.7)
    rig = synth.Rig(13, 40.0, 4.0, 50.0)
    scene = synth.uniform_scene(1500, 77)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    plan = lfd.Plan(panel, tile=tile, views_per_cluster=4)
    img, _ = plan.render(lfd.scene_to_device(scene), cams)
    proj = oracle.project(scene, cams, panel.width, panel.height, 4)
    ref, lo, hi = oracle.render_bracket(proj, oracle.view_index(panel), 4, mode=1, tile=tile)
    assert_render_matches(img.cpu().numpy(), ref, lo, hi, f"ragged {tile}")
    plan.close()


def test_edge_cases(tiny):
    w, scene, cams = tiny
    bg = (0.1, 0.2, 0.3)
    # no Gaussians: background everywhere
    plan = lfd.Plan(w.panel, views_per_cluster=8, bg=bg)
    empty = {k: v[:0] for k, v in scene.items()}
    img, st = plan.render(lfd.scene_to_device(empty), cams)
    assert st["num_pairs"] == 0
    np.testing.assert_array_equal(img.cpu().numpy(), np.broadcast_to(np.float32(bg), img.shape))
    # everything behind every camera
    behind = dict(scene)
    behind["means"] = (scene["means"] * 0.01 + np.float32([0, 0, -50])).astype(np.float32)
    img, st = plan.render(lfd.scene_to_device(behind), cams)
    assert st["num_pairs"] == 0
    np.testing.assert_array_equal(img.cpu().numpy(), np.broadcast_to(np.float32(bg), img.shape))
    plan.close()
    # one view (plain 3DGS) and one cluster holding every view
    for panel, c, nv in ((synth.Panel(128, 72, 1, 0.2, 5.0), 1, 1),
                         (synth.Panel(128, 72, 6, 0.2, 5.0), 8, 6)):
        rig = synth.Rig(nv, 20.0, 4.0, 50.0)
        cm = synth.arc_cameras(rig, panel.width, panel.height)
        sc = synth.uniform_scene(800, 5)
        plan = lfd.Plan(panel, views_per_cluster=c)
        img, _ = plan.render(lfd.scene_to_device(sc), cm)
        proj = oracle.project(sc, cm, panel.width, panel.height, c)
        ref, lo, hi = oracle.render_bracket(proj, oracle.view_index(panel), c, mode=1)
        assert_render_matches(img.cpu().numpy(), ref, lo, hi, f"N={nv} C={c}")
        plan.close()


@pytest.mark.parametrize("c", [1, 8])
def test_without_remap_gives_the_same_image(tiny, c):
    # the ablation "w/o remap" (threads in raster order, each walking its own
    # list from global memory) computes the very same per-entry arithmetic
    w, scene, cams = tiny
    s = lfd.scene_to_device(scene)
    a, _ = lfd.Plan(w.panel, views_per_cluster=c).render(s, cams)
    b, _ = lfd.Plan(w.panel, views_per_cluster=c, remap=False).render(s, cams)
    assert torch.equal(a, b)


def test_large_tiles_give_the_same_image(tiny):
    # tiles of up to 1024 pixels (a run of one cluster then holds up to 3072
    # subpixels): the image does not depend on the tile shape, and the
    # full-frame baseline of such a plan (its tile cut to 512 pixels) neither
    w, scene, cams = tiny
    s = lfd.scene_to_device(scene)
    base = lfd.Plan(w.panel, tile=(16, 16), views_per_cluster=8)
    want, _ = base.render(s, cams)
    want = want.clone()
    want_ff, _ = base.render_fullframe(s, cams)
    want_ff = want_ff.clone()
    for tile in [(32, 24), (32, 32), (64, 16)]:
        plan = lfd.Plan(w.panel, tile=tile, views_per_cluster=8)
        got, _ = plan.render(s, cams)
        assert torch.equal(got, want), tile
        ff, _ = plan.render_fullframe(s, cams)
        assert torch.equal(ff, want_ff), tile
        plan.close()
    base.close()


def test_fullframe_baseline_matches_oracle_and_subpixel_path(tiny):
    # every view rendered whole, then interlaced: the oracle's full-frame
    # renderer, and the subpixel path with one view per cluster
    w, scene, cams = tiny
    s = lfd.scene_to_device(scene)
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    ff, st = plan.render_fullframe(s, cams)
    ff = ff.cpu().numpy()
    proj1 = oracle.project(scene, cams, w.panel.width, w.panel.height, 1)
    V = oracle.view_index(w.panel)
    ref, lo, hi = oracle.render_bracket(proj1, V, 1, mode=1)
    assert_render_matches(ff, ref, lo, hi, "full-frame")
    np.testing.assert_array_equal(oracle.render_fullframe(proj1, V, crop=(0, 0, 64, 48)),
                                  ref[:48, :64])
    sub, _ = lfd.Plan(w.panel, views_per_cluster=1).render(s, cams)
    np.testing.assert_allclose(ff, sub.cpu().numpy(), rtol=0, atol=2e-5)
    plan.close()


@pytest.mark.parametrize("dt", ["float16", "bfloat16"])
def test_half_precision_attributes(tiny, dt):
    # Scales, rotations, opacity and SH stored in FP16 / BF16 (means FP32):
    # the kernel error is measured against the FP64 oracle fed the
    # dequantised attributes (exact in FP32) and must meet the bar; the
    # storage error against the FP32 originals is only bounded loosely.
    w, scene, cams = tiny
    s = lfd.scene_to_device(scene, attr_dtype=getattr(torch, dt))
    assert s["sh"].dtype == getattr(torch, dt) and s["means"].dtype == torch.float32
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    img, _ = plan.render(s, cams)
    got = img.cpu().numpy()
    deq = {k: v.float().cpu().numpy() for k, v in s.items()}
    V = oracle.view_index(w.panel)
    proj = oracle.project(deq, cams, w.panel.width, w.panel.height, 8)
    ref, lo, hi = oracle.render_bracket(proj, V, 8, mode=1)
    assert_render_matches(got, ref, lo, hi, f"{dt} attributes")
    proj32 = oracle.project(scene, cams, w.panel.width, w.panel.height, 8)
    ref32, _ = oracle.render(proj32, V, 8, mode=1)
    assert image_metrics(got, ref32)["psnr"] > 35
    plan.close()


def test_deterministic(tiny):
    w, scene, cams = tiny
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    s = lfd.scene_to_device(scene)
    a, _ = plan.render(s, cams)
    a = a.clone()
    b, _ = plan.render(s, cams)
    assert torch.equal(a, b)
    plan.close()


@pytest.mark.parametrize("remap", [True, False])
def test_host_entry_point_matches_device(tiny, remap):
    # the host entry point copies the Gaussians up in chunks, projecting each
    # as it lands, and (remapped blend) the image back in bands of tile rows
    w, scene, cams = tiny
    plan = lfd.Plan(w.panel, views_per_cluster=8, remap=remap)
    dev, _ = plan.render(lfd.scene_to_device(scene), cams)
    host_scene = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in scene.items()}
    out = torch.empty(dev.shape, dtype=torch.float32).pin_memory()
    plan.render_host(host_scene, cams, out)
    assert torch.equal(out, dev.cpu())
    plan.close()


def test_host_pipelined_frames_match_device(tiny):
    # several frames queued with lfd_render_host_async before one wait: each
    # frame's upload runs under the previous frame's blend and the plan
    # alternates two sets of device buffers; one frame has fewer Gaussians
    w, scene, cams = tiny
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    scenes = [scene,
              dict(scene, opacities=(scene["opacities"] * 0.5).astype(np.float32)),
              {k: v[: len(v) // 2] for k, v in scene.items()},
              dict(scene, means=(scene["means"] + 0.05).astype(np.float32))]
    refs = [plan.render(lfd.scene_to_device(sc), cams)[0].cpu() for sc in scenes]
    hosts = [{k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in sc.items()}
             for sc in scenes]
    outs = [torch.full(refs[0].shape, -1.0, dtype=torch.float32).pin_memory() for _ in scenes]
    for _ in range(2):
        for h, o in zip(hosts, outs):
            plan.render_host_async(h, cams, o)
        plan.render_host_wait()
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert torch.equal(o, r), i
        for o in outs:
            o.fill_(-1.0)
    plan.close()


@pytest.mark.parametrize("height,count", [(32, 2001), (144, 3), (16, 0)])
def test_host_entry_point_ragged(height, count):
    # fewer tile rows than bands, Gaussian counts not divisible by the chunk
    # count (or below it, or zero), FP16 attributes from pageable memory
    panel = synth.Panel(96, height, 8, math.tan(0.2), 4.5, 0.0)
    rig = synth.Rig(8, 40.0, 4.0, 50.0)
    cams = synth.arc_cameras(rig, panel.width, panel.height)
    scene = synth.uniform_scene(count, 9, half_extent=0.8)
    plan = lfd.Plan(panel, views_per_cluster=8)
    dev, _ = plan.render(lfd.scene_to_device(scene, attr_dtype=torch.float16), cams)
    host_scene = {k: (torch.from_numpy(np.ascontiguousarray(v)) if k == "means"
                      else torch.from_numpy(np.ascontiguousarray(v)).to(torch.float16))
                  for k, v in scene.items()}
    out = torch.full(dev.shape, -1.0, dtype=torch.float32)
    plan.render_host(host_scene, cams, out)
    assert torch.equal(out, dev.cpu())
    plan.close()


def test_invalid_arguments(tiny):
    w, scene, cams = tiny
    with pytest.raises(lfd.LFDError) as e:
        lfd.Plan(synth.Panel(0, 10, 8, 0.1, 4.0))
    assert e.value.status == lfd.LFD_ERR_INVALID
    with pytest.raises(lfd.LFDError):
        lfd.Plan(w.panel, tile=(64, 64))
    with pytest.raises(lfd.LFDError):
        lfd.Plan(w.panel, views_per_cluster=0)
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    with pytest.raises(lfd.LFDError) as e:
        plan.render(lfd.scene_to_device(scene), cams[:3])
    assert e.value.status == lfd.LFD_ERR_INVALID
    plan.close()


@pytest.fixture(scope="module")
def paper4k_oracle():
    w = synth.WORKLOADS["paper4k"]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    proj = oracle.project(scene, cams, w.panel.width, w.panel.height, 8)
    return w, scene, cams, proj, oracle.view_index(w.panel)


@pytest.mark.slow
@pytest.mark.parametrize("tile", [(32, 16), (16, 16), (32, 24)])
def test_paper4k_sampled_crops(paper4k_oracle, tile):
    # The paper-scale workload at full size, in the launch configurations the
    # benchmark times (32x16 is the tile its autotuner picks); the oracle
    # recomputes sampled crops by definition.
    w, scene, cams, proj, V = paper4k_oracle
    c = 8
    plan = lfd.Plan(w.panel, tile=tile, views_per_cluster=c)
    img, st = plan.render(lfd.scene_to_device(scene), cams)
    got = img.cpu().numpy()
    assert st["num_pairs"] > 10_000_000
    # crops: the densest region, the panel centre, random places, the edge
    dens = np.clip(got, 0, 1).sum(-1)
    yy, xx = np.unravel_index(np.argmax(dens), dens.shape)
    rng = np.random.default_rng(8)
    crops = [(min(xx // 16, 239) * 16, min(yy // 16, 134) * 16, 16, 16), (3824, 2144, 16, 16),
             (1664, 952, 512, 256)]  # the central 512x256 crop holds the densest blobs
    crops += [(int(rng.integers(0, 240)) * 16, int(rng.integers(0, 135)) * 16, 16, 16)
              for _ in range(3)]
    for x0, y0, cw, ch in crops:
        crop = (x0, y0, x0 + cw, y0 + ch)
        ref, lo, hi = oracle.render_bracket(proj, V, c, crop=crop, mode=1)
        assert_render_matches(got[y0:y0 + ch, x0:x0 + cw], ref, lo, hi, f"crop {crop}")
    plan.close()


def test_depth_first_lists_equal_eq11_key_sort_on_4k():
    # the paper4k panel at full size (300k Gaussians, 32x16 tiles): sorting the
    # depths once and the emitted pairs by their tile bits gives the same list,
    # ranges and image as sorting the 64-bit keys of Eq. 11
    w = synth.WORKLOADS["paper4k"]
    scene = lfd.scene_to_device(synth.scene_for(w, 300_000))
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    got = {}
    for mode in (lfd.SORT_DEPTH_FIRST, lfd.SORT_KEY64):
        plan = lfd.Plan(w.panel, tile=(32, 16), views_per_cluster=8, sort_mode=mode)
        img, st = plan.render(scene, cams)
        lst, ranges, _ = plan.lists(st["num_pairs"])
        got[mode] = (img.cpu(), lst, ranges, st["num_pairs"])
        plan.close()
    a, b = got[lfd.SORT_DEPTH_FIRST], got[lfd.SORT_KEY64]
    assert a[3] == b[3] > 10_000_000
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[1], b[1])
    assert torch.equal(a[0], b[0])
