"""Autotuner over the tile shape.

The tile shape changes how many Gaussian-(tile, cluster) pairs the key
generation emits and sorts (smaller tiles: more pairs, shorter lists) and how
many subpixels one blend warp owns; it does not change the image: every
subpixel meets the same Gaussians in the same depth order whatever the tile
(the paper gives 16x16 only as an example tile, Sec. 4.2). Tiles may hold up
to 1024 pixels; the default candidates span the batching range 8x8..32x16,
and callers pass larger shapes (32x24, 32x32) where the panel favours them. The plan's subpixels_per_thread option is still accepted as
a candidate dimension, but the warp-per-run blend ignores it, so the default
candidate list holds only 0. The tuner renders a few frames
with each candidate plan on the caller's scene and cameras, times them with
CUDA events on the rendering stream, checks every candidate's image against
the first one's, and returns the fastest configuration.

    python -m paper_2605_04509_gb300.autotune --workload paper4k
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, Iterable, List, Optional, Tuple

TILES: Tuple[Tuple[int, int], ...] = ((8, 8), (16, 8), (16, 16), (32, 8), (32, 16))
SUBPIXELS_PER_THREAD: Tuple[int, ...] = (0,)


def time_plan(plan, scene, cams, out, frames: int, warmup: int) -> float:
    """Mean milliseconds per lfd_render frame, CUDA events on the stream."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.render(scene, cams, out, stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(frames):
        plan.render(scene, cams, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / frames


def tune(panel, scene, cams, views_per_cluster: int = 8,
         tiles: Iterable[Tuple[int, int]] = TILES,
         subpixels_per_thread: Iterable[int] = SUBPIXELS_PER_THREAD,
         frames: int = 3, warmup: int = 2, tol: float = 2e-3) -> Dict:
    """Time every (tile, subpixels_per_thread) candidate on this scene.

    scene: device scene dict (lfd.scene_to_device); cams: [N, 16] float32.
    Returns {"best": {...}, "results": [...]}; each result has the tile, the
    staging setting, ms per frame, the pair count P and the max |difference|
    of its clamped image from the first candidate's."""
    import torch
    from . import lfd
    out = torch.empty((panel.height, panel.width, 3), dtype=torch.float32, device="cuda")
    ref = None
    results: List[Dict] = []
    for tile in tiles:
        for spt in subpixels_per_thread:
            try:
                plan = lfd.Plan(panel, tile=tuple(tile), views_per_cluster=views_per_cluster,
                                subpixels_per_thread=spt)
            except lfd.LFDError:
                continue
            try:
                _, st = plan.render(scene, cams, out)
                ms = time_plan(plan, scene, cams, out, frames, warmup)
            except lfd.LFDError as e:  # e.g. more pairs than 2^32 with small tiles
                results.append({"tile": list(tile), "subpixels_per_thread": spt,
                                "skipped": str(e)})
                continue
            finally:
                plan.close()
            img = out.clamp(0, 1)
            if ref is None:
                ref = img.clone()
                diff = 0.0
            else:
                diff = float((img - ref).abs().max())
            results.append({"tile": list(tile), "subpixels_per_thread": spt, "ms": ms,
                            "pairs": int(st["num_pairs"]), "max_diff": diff})
            if diff > tol:
                raise RuntimeError(f"tile {tile} / {spt}: image differs by {diff}")
    timed_ok = [r for r in results if "ms" in r]
    if not timed_ok:
        raise RuntimeError("no candidate configuration could render this scene")
    best = min(timed_ok, key=lambda r: r["ms"])
    return {"best": best, "results": results}


def cached_tune(cache_path: Optional[str], key: str, **kw) -> Dict:
    """tune() with a JSON cache keyed by `key` (e.g. panel and scene size)."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        return cache[key]
    res = tune(**kw)
    if cache_path:
        cache[key] = res
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return res


def main(argv=None) -> int:
    from . import lfd, synth
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="paper4k", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--gaussians", type=int, default=0)
    ap.add_argument("--views-per-cluster", type=int, default=8)
    ap.add_argument("--frames", type=int, default=5)
    args = ap.parse_args(argv)
    w = synth.WORKLOADS[args.workload]
    scene = lfd.scene_to_device(synth.scene_for(w, args.gaussians or None))
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    t0 = time.perf_counter()
    res = tune(w.panel, scene, cams, views_per_cluster=args.views_per_cluster, frames=args.frames)
    res["workload"] = args.workload
    res["seconds"] = time.perf_counter() - t0
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
