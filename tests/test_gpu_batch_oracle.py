"""Batched rendering against the FP64 oracle directly (not only against the
single-scene frames): one lfd_batch_render of three scenes with mixed panels
- the tiny panel, a ragged 250x141 panel with 13 views and a K_offset, and
the paper-scale 4K / 45-view panel with 1M Gaussians in FP16 - each scene's
image compared element by element with the oracle's definition (the tiny and
ragged panels whole, the 4K panel on a 256x256 crop and an edge crop), under
the bracket reading of the 1/255 threshold."""
import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth

from .helpers import assert_render_matches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_04509_gb300 import lfd  # noqa: E402

RAGGED = synth.Panel(250, 141, 13, 0.2027, 5.3, 0.7)
RAGGED_RIG = synth.Rig(13, 30.0, 4.0, 50.0)


def test_batch_scenes_match_oracle():
    tiny = synth.WORKLOADS["tiny"]
    p4k = synth.WORKLOADS["paper4k"]
    specs = [
        # (panel, rig, host scene, views per cluster, tile, attribute dtype)
        (tiny.panel, tiny.rig, synth.scene_for(tiny), 8, (16, 16), torch.float32),
        (RAGGED, RAGGED_RIG, synth.uniform_scene(2500, 101), 4, (16, 16), torch.float32),
        (p4k.panel, p4k.rig, synth.scene_for(p4k), 8, (32, 16), torch.float16),
    ]
    plans, scenes, cams, hosts = [], [], [], []
    for panel, rig, host, c, tile, dt in specs:
        plans.append(lfd.Plan(panel, tile=tile, views_per_cluster=c))
        scenes.append(lfd.scene_to_device(host, attr_dtype=dt))
        cams.append(synth.arc_cameras(rig, panel.width, panel.height))
        # the oracle sees exactly the stored (dequantised) attributes
        hosts.append({k: (v if k == "means" or dt == torch.float32
                          else v.astype(np.float16).astype(np.float32)) for k, v in host.items()})
    pairs = []
    for pl, sc, cm in zip(plans, scenes, cams):
        _, st = pl.render(sc, cm)
        pairs.append(int(st["num_pairs"]))
    batch = lfd.Batch(plans)
    batch.reserve([sc["means"].shape[0] for sc in scenes], sum(pairs) + 1024)
    outs = batch.render(scenes, cams)
    assert batch.status() == sum(pairs)
    for (panel, rig, _h, c, tile, _dt), host, cm, out in zip(specs, hosts, cams, outs):
        got = out.cpu().numpy().astype(np.float64)
        V = oracle.view_index(panel)
        proj = oracle.project(host, cm, panel.width, panel.height, c)
        if panel.width * panel.height > 1_000_000:
            cx, cy = panel.width // 2, panel.height // 2
            crops = [(cx - 128, cy - 128, cx + 128, cy + 128),
                     (panel.width - 192, 0, panel.width, 128)]
        else:
            crops = [(0, 0, panel.width, panel.height)]
        for cr in crops:
            ref, lo, hi = oracle.render_bracket(proj, V, c, crop=cr, mode=1, tile=tile)
            assert_render_matches(got[cr[1]:cr[3], cr[0]:cr[2]], ref, lo, hi,
                                  what=f"batched {panel.width}x{panel.height} crop {cr}")
    batch.close()
    for pl in plans:
        pl.close()
