"""Ablation of the two components (the paper's ablation study, T3, with the
stage breakdown of T5/T6): cross-view attribute reuse on/off (clusters of 8
views vs 1) and view-coherent remapping on/off, on one synthetic workload.

    python -m paper_2605_04509_gb300.ablation [--workload paper4k] [--frames 20] [--tile 32x16]
    python -m paper_2605_04509_gb300.ablation --reuse [--workload paper4k]

Prints one JSON line per configuration and a markdown table. Every
configuration renders through the C ABI; the images of the remap on/off pairs
are checked to be identical. --reuse reports the image-quality side of
attribute reuse (Table 1's trend): PSNR of the |V_k| = 2, 4, 8, 16 renders
against the exact |V_k| = 1 render of the same scene, over the whole panel.
"""
from __future__ import annotations

import argparse
import hashlib
import json

import numpy as np


def run(workload: str = "paper4k", frames: int = 20, warmup: int = 3, tile=(32, 16)):
    import torch

    from . import lfd, synth

    w = synth.WORKLOADS[workload]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    s = lfd.scene_to_device(scene)
    out = torch.empty((w.panel.height, w.panel.width, 3), dtype=torch.float32, device="cuda")
    rows = []
    for c, remap, name in ((1, False, "w/o reuse, w/o remap"), (1, True, "w/o reuse"),
                           (8, False, "w/o remap"), (8, True, "ours")):
        plan = lfd.Plan(w.panel, tile=tuple(tile), views_per_cluster=c, remap=remap)
        for _ in range(warmup):
            plan.render(s, cams, out)
        plan.set_flags(lfd.FLAG_COUNT_EVALS)
        _, st = plan.render(s, cams, out)
        plan.set_flags(lfd.FLAG_STAGE_TIMING)
        plan.stage_totals(reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(frames):
            plan.render(s, cams, out)
        e1.record()
        torch.cuda.synchronize()
        tot = plan.stage_totals(reset=True)
        ms = e0.elapsed_time(e1) / frames
        row = {"config": name, "views_per_cluster": c, "remap": remap, "tile": list(tile),
               "fps": 1000.0 / ms,
               "ms_per_frame": ms, "pairs": st["num_pairs"], "visits": st["num_visits"],
               "evals": st["num_evals"],
               "image_sha256": hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest()[:16]}
        for k in ("ms_project", "ms_keygen", "ms_sort", "ms_blend"):
            row[k] = tot[k] / max(tot["frames"], 1)
        rows.append(row)
        print(json.dumps(row), flush=True)
        plan.close()
    assert rows[0]["image_sha256"] == rows[1]["image_sha256"], "remap changed the image (C=1)"
    assert rows[2]["image_sha256"] == rows[3]["image_sha256"], "remap changed the image (C=8)"
    print("\n| config | frames/s | ms/frame | project | keygen | sort | blend | pairs | evaluations |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['config']} | {r['fps']:.1f} | {r['ms_per_frame']:.2f} | {r['ms_project']:.2f} | "
              f"{r['ms_keygen']:.2f} | {r['ms_sort']:.2f} | {r['ms_blend']:.2f} | "
              f"{r['pairs'] / 1e6:.1f}M | {r['evals'] / 1e9:.2f}G |")
    return rows


def reuse_quality(workload: str = "paper4k", sizes=(2, 4, 8, 16), tile=(32, 16)):
    """PSNR, max |err| and share of subpixels off by more than 1/255 of the
    |V_k| = c renders against the |V_k| = 1 render (clamped to [0, 1])."""
    import math

    import torch

    from . import lfd, synth

    w = synth.WORKLOADS[workload]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    s = lfd.scene_to_device(scene)
    imgs = {}
    for c in (1,) + tuple(sizes):
        plan = lfd.Plan(w.panel, tile=tuple(tile), views_per_cluster=c)
        out = torch.empty((w.panel.height, w.panel.width, 3), dtype=torch.float32, device="cuda")
        plan.render(s, cams, out)
        torch.cuda.synchronize()
        imgs[c] = out.clamp(0, 1)
        plan.close()
    rows = []
    for c in sizes:
        err = (imgs[c] - imgs[1]).abs()
        mse = float((err.double() ** 2).mean())
        row = {"views_per_cluster": c, "psnr_db_vs_c1": float("inf") if mse == 0 else 10 * math.log10(1 / mse),
               "max_err_vs_c1": float(err.max()), "frac_off_1_255": float((err > 1 / 255).float().mean())}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print("\n| |V_k| | PSNR vs |V_k| = 1 | max err | off by > 1/255 |")
    print("|---|---|---|---|")
    for r in rows:
        print(f"| {r['views_per_cluster']} | {r['psnr_db_vs_c1']:.2f} dB | {r['max_err_vs_c1']:.3f} | "
              f"{r['frac_off_1_255']:.2%} |")
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--workload", default="paper4k")
    ap.add_argument("--frames", type=int, default=20)
    ap.add_argument("--tile", default="32x16")
    ap.add_argument("--reuse", action="store_true", help="image quality of attribute reuse vs |V_k|")
    args = ap.parse_args()
    np.set_printoptions(precision=3)
    tile = tuple(int(v) for v in args.tile.split("x"))
    if args.reuse:
        reuse_quality(args.workload, tile=tile)
    else:
        run(args.workload, args.frames, tile=tile)


if __name__ == "__main__":
    main()
