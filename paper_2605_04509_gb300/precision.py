"""FP16 / BF16 attribute storage on the precision workload (north-star
precision configuration): 3M Gaussians, 100 views over 50 degrees, a
7680x4320 panel (slant 0.18 rad, pitch 6.1 subpixels), clusters of 8 views.

    python -m paper_2605_04509_gb300.precision [--frames 5] [--crop 512]

For each storage type of scales, rotations, opacity and SH (means stay FP32;
the 2D-covariance inverse, the blend and the transmittance product are FP32)
it prints frames/s and, on the central crop, the error against the FP64
oracle fed the dequantised attributes (the kernel's error) and against the
FP64 oracle on the FP32 originals (kernel + storage error): max |err|, the
share of subpixels off by more than 1/255, PSNR.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def _metrics(got, ref, lo=None, hi=None):
    g, r = np.clip(got, 0, 1), np.clip(ref, 0, 1)
    err = np.abs(g - r)
    mse = float((err ** 2).mean())
    out = {"max_err": float(err.max()), "frac_off_1_255": float((err > 1 / 255).mean()),
           "psnr_db": float("inf") if mse == 0 else 10 * math.log10(1 / mse)}
    if lo is not None:
        # where the definition itself jumps at the 1/255 skip threshold (the
        # oracle rendered at 1/255 * (1 -/+ 1e-3) differs by more than 1e-3)
        a, b = np.clip(lo, 0, 1), np.clip(hi, 0, 1)
        jump = (np.maximum(np.maximum(r, a), b) - np.minimum(np.minimum(r, a), b)) > 1e-3
        out["max_err_outside_threshold_jumps"] = float(err[~jump].max()) if (~jump).any() else 0.0
        out["threshold_jump_subpixels"] = int(jump.sum())
    return out


def run(frames: int = 5, crop_px: int = 512, gaussians: int = 0):
    import torch

    import oracle

    from . import lfd, synth

    w = synth.WORKLOADS["precision8k"]
    scene = synth.scene_for(w, gaussians or None)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    c = 8
    cw = min(crop_px, w.panel.width)
    ch = min(crop_px, w.panel.height)
    x0, y0 = (w.panel.width - cw) // 2, (w.panel.height - ch) // 2
    crop = (x0, y0, x0 + cw, y0 + ch)
    V = oracle.view_index(w.panel)
    proj32 = oracle.project(scene, cams, w.panel.width, w.panel.height, c)
    ref32, _ = oracle.render(proj32, V, c, crop=crop, mode=1, tile=(32, 16))
    del proj32
    # 32x16 tiles at 8K keep the Gaussian-tile pair count below 2^32
    plan = lfd.Plan(w.panel, tile=(32, 16), views_per_cluster=c)
    rows = []
    for name, dt in (("fp32", torch.float32), ("fp16", torch.float16), ("bf16", torch.bfloat16)):
        s = lfd.scene_to_device(scene, attr_dtype=dt)
        out = torch.empty((w.panel.height, w.panel.width, 3), dtype=torch.float32, device="cuda")
        for _ in range(2):
            _, st = plan.render(s, cams, out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(frames):
            plan.render(s, cams, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / frames
        got = out[crop[1]:crop[3], crop[0]:crop[2]].cpu().numpy().astype(np.float64)
        deq = {k: v.float().cpu().numpy() for k, v in s.items()}
        proj = oracle.project(deq, cams, w.panel.width, w.panel.height, c)
        ref, lo, hi = oracle.render_bracket(proj, V, c, crop=crop, mode=1, tile=(32, 16))
        del proj
        row = {"attributes": name, "fps": 1000.0 / ms, "ms_per_frame": ms, "pairs": st["num_pairs"],
               "attr_bytes_per_gaussian": 12 + (4 if name == "fp32" else 2) * (3 + 4 + 1 + 48),
               "vs_dequantised_oracle": _metrics(got, ref, lo, hi), "vs_fp32_oracle": _metrics(got, ref32),
               "crop": list(crop)}
        rows.append(row)
        print(json.dumps(row), flush=True)
        del s, out
    plan.close()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--frames", type=int, default=5)
    ap.add_argument("--crop", type=int, default=512)
    ap.add_argument("--gaussians", type=int, default=0)
    args = ap.parse_args()
    run(args.frames, args.crop, args.gaussians)


if __name__ == "__main__":
    main()
