"""Batched rendering of many scenes with mixed panels (the batching
workload): 16 seeded scenes (seeds 100-115) of 200k-3M Gaussians (log-
uniform), panels assigned round-robin from 1536x2048 / 48 views,
3840x2160 / 45 views and 7680x4320 / 100 views, all attributes in FP16.

    python -m paper_2605_04509_gb300.batching [--frames 3] [--scenes 16] [--sizes 200000,3000000]
    python -m paper_2605_04509_gb300.batching --probe --tiles 16x16,32x16,32x16

(--probe: only the batch, with the given tile per panel and no tuning or
single-scene frames, rendered --frames times; for profiler launch lists.)

Per panel the autotuner picks the tile shape on that panel's first scene. Scenes are grouped into as few batches as the 2^32 pair limit allows
(one for these sizes); each batch is one lfd_batch_render - one persistent
blend launch - captured into a CUDA graph. It prints, as JSON lines, the
tuning tables and the throughput of three schedules of the same work:
single-scene frames one after the other (lfd_render, with its host
read-back per scene), the batch launched directly, and the batch replayed
from the CUDA graph; every batched image is checked bit for bit against the
scene's single-scene frame.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import synth

PANELS = (
    ("1536x2048/48", synth.Panel(1536, 2048, 48, math.tan(0.2), 4.6, 0.0), synth.Rig(48, 35.0, 30.0, 50.0)),
    ("3840x2160/45", synth.WORKLOADS["paper4k"].panel, synth.WORKLOADS["paper4k"].rig),
    ("7680x4320/100", synth.WORKLOADS["precision8k"].panel, synth.WORKLOADS["precision8k"].rig),
)
TILES = ((16, 16), (32, 16), (32, 8), (16, 8))
MAX_PAIRS = (1 << 32) - 2


def scene_sizes(n: int, lo: int = 200_000, hi: int = 3_000_000):
    """Gaussian count of scene s: log-uniform in [lo, hi] from seed 100 + s."""
    out = []
    for s in range(n):
        u = np.random.default_rng(100 + s).uniform()
        out.append(int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    return out


def group_scenes(pairs, max_pairs: int = MAX_PAIRS, max_scenes: int = 16):
    """Scenes (in order) grouped into as few batches as the pair limit and the
    per-batch scene limit allow; a scene above the limit alone still gets a
    batch of its own (its render then reports the capacity error)."""
    groups, cur, cur_p = [], [], 0
    for s, p in enumerate(pairs):
        if cur and (cur_p + p > max_pairs or len(cur) == max_scenes):
            groups.append(cur)
            cur, cur_p = [], 0
        cur.append(s)
        cur_p += p
    if cur:
        groups.append(cur)
    return groups


def timed(fn, frames: int) -> float:
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(frames):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / frames


def run(frames: int = 3, n_scenes: int = 16, tune_frames: int = 2, lo: int = 200_000,
        hi: int = 3_000_000):
    import torch

    from . import autotune, lfd

    sizes = scene_sizes(n_scenes, lo, hi)
    panel_of = [s % len(PANELS) for s in range(n_scenes)]
    t0 = time.perf_counter()
    scenes = [lfd.scene_to_device(synth.mixture_scene(sizes[s], 100 + s), attr_dtype=torch.float16)
              for s in range(n_scenes)]
    cams = [synth.arc_cameras(PANELS[p][2], PANELS[p][1].width, PANELS[p][1].height)
            for p in range(len(PANELS))]
    t_gen = time.perf_counter() - t0

    # tile shape per panel, on the panel's first scene
    tiles = {}
    for p, (name, panel, _rig) in enumerate(PANELS):
        first = panel_of.index(p)
        res = autotune.tune(panel, scenes[first], cams[p], views_per_cluster=8, tiles=TILES,
                            subpixels_per_thread=(0,), frames=tune_frames, warmup=1)
        tiles[p] = tuple(res["best"]["tile"])
        print(json.dumps({"autotune_panel": name, "scene": first, "gaussians": sizes[first],
                          "chosen_tile": list(tiles[p]),
                          "ms_per_frame": {f"{r['tile'][0]}x{r['tile'][1]}": round(r["ms"], 3)
                                           for r in res["results"] if "ms" in r}}), flush=True)

    def make_plans(spt):
        return {p: lfd.Plan(PANELS[p][1], tile=tiles[p], views_per_cluster=8,
                            subpixels_per_thread=spt) for p in range(len(PANELS))}

    # single-scene reference frames (and their pair counts)
    plans = make_plans(0)
    refs, pairs = [], []
    for s in range(n_scenes):
        img, st = plans[panel_of[s]].render(scenes[s], cams[panel_of[s]])
        refs.append(img.clone())
        pairs.append(int(st["num_pairs"]))
    torch.cuda.synchronize()

    def sequential():
        for s in range(n_scenes):
            plans[panel_of[s]].render(scenes[s], cams[panel_of[s]], refs_out[s])

    refs_out = [torch.empty_like(r) for r in refs]
    sequential()
    ms_seq = timed(sequential, frames)

    # group scenes into batches below the pair limit (in scene order)
    groups = group_scenes(pairs)

    def build(spt):
        pl = make_plans(spt)
        batches = []
        for g in groups:
            b = lfd.Batch([pl[panel_of[s]] for s in g])
            b.reserve([sizes[s] for s in g], min(sum(pairs[s] for s in g) + 1024, MAX_PAIRS))
            outs = [torch.empty_like(refs[s]) for s in g]
            batches.append((b, g, outs))
        return pl, batches

    def run_batches(batches):
        for b, g, outs in batches:
            b.render([scenes[s] for s in g], [cams[panel_of[s]] for s in g], outs)

    spt = 0  # the warp-per-run blend has no staging-depth choice
    pl, batches = build(spt)
    run_batches(batches)
    total_pairs = 0
    for b, _, _ in batches:
        total_pairs += b.status()
    ms_direct = timed(lambda: run_batches(batches), frames)
    for b, _, _ in batches:
        b.status()
    # capture every batch of the frame into one CUDA graph
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        run_batches(batches)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        run_batches(batches)
    for _, _, outs in batches:
        for o in outs:
            o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for b, _, _ in batches:
        b.status()
    identical = all(torch.equal(o, refs[s]) for _, g, outs in batches for s, o in zip(g, outs))
    ms_graph = timed(graph.replay, frames)
    for b, _, _ in batches:
        b.status()

    subpixels = sum(PANELS[panel_of[s]][1].subpixels for s in range(n_scenes))
    line = {
        "workload": f"{n_scenes} scenes, {lo}-{hi} Gaussians (log-uniform, seeds 100-{99 + n_scenes}), "
                    "panels round-robin " + ", ".join(p[0] for p in PANELS) + ", FP16 attributes, "
                    "|V_k| = 8",
        "gaussians": sizes, "panels": [PANELS[p][0] for p in panel_of], "pairs": pairs,
        "tiles": {PANELS[p][0]: f"{tiles[p][0]}x{tiles[p][1]}" for p in tiles},
        "subpixels_per_thread": spt, "batches": [len(g) for g in groups],
        "images_identical_to_single_scene_frames": identical,
        "sequential": {"ms_per_round": ms_seq, "scenes_per_s": n_scenes * 1000.0 / ms_seq,
                       "subpixels_per_s": subpixels * 1000.0 / ms_seq},
        "batched": {"ms_per_round": ms_direct, "scenes_per_s": n_scenes * 1000.0 / ms_direct,
                    "subpixels_per_s": subpixels * 1000.0 / ms_direct},
        "batched_graph": {"ms_per_round": ms_graph, "scenes_per_s": n_scenes * 1000.0 / ms_graph,
                          "subpixels_per_s": subpixels * 1000.0 / ms_graph},
        "total_pairs": total_pairs, "scene_generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)
    for b, _, _ in batches:
        b.close()
    return line


def probe(frames: int, n_scenes: int, tiles):
    """Build the batch with fixed tiles (one per panel) and render it."""
    import torch

    from . import lfd

    sizes = scene_sizes(n_scenes)
    panel_of = [s % len(PANELS) for s in range(n_scenes)]
    scenes = [lfd.scene_to_device(synth.mixture_scene(sizes[s], 100 + s), attr_dtype=torch.float16)
              for s in range(n_scenes)]
    cams = [synth.arc_cameras(PANELS[p][2], PANELS[p][1].width, PANELS[p][1].height)
            for p in range(len(PANELS))]
    plans = {p: lfd.Plan(PANELS[p][1], tile=tiles[p], views_per_cluster=8) for p in range(len(PANELS))}
    batch = lfd.Batch([plans[panel_of[s]] for s in range(n_scenes)])
    batch.reserve(sizes, MAX_PAIRS)
    outs = batch.images()
    for it in range(frames):
        batch.render(scenes, [cams[panel_of[s]] for s in range(n_scenes)], outs)
        print(json.dumps({"frame": it, "pairs": batch.status()}), flush=True)
    batch.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--scenes", type=int, default=16)
    ap.add_argument("--probe", action="store_true")
    ap.add_argument("--tiles", default="16x16,32x16,32x16")
    ap.add_argument("--sizes", default="200000,3000000",
                    help="lo,hi: Gaussian counts drawn log-uniform in [lo, hi]")
    args = ap.parse_args()
    lo, hi = (int(v) for v in args.sizes.split(","))
    if args.probe:
        tiles = [tuple(int(v) for v in t.split("x")) for t in args.tiles.split(",")]
        probe(args.frames, args.scenes, tiles)
    else:
        run(args.frames, args.scenes, lo=lo, hi=hi)


if __name__ == "__main__":
    main()
