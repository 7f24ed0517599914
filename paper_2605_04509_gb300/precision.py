"""FP16 / BF16 attribute storage on the precision workload: 3M Gaussians,
100 views over 50 degrees, a 7680x4320 panel (slant 0.18 rad, pitch 6.1 subpixels), clusters of 8 views.

    python -m paper_2605_04509_gb300.precision [--frames 5]

For each storage type of scales, rotations, opacity and SH (means stay FP32;
the 2D-covariance inverse, the blend and the transmittance product are FP32)
it prints frames/s, attribute bytes per Gaussian and the storage error: the
FP16/BF16 image against the FP32-attribute image of the same renderer (max
|err|, share of subpixels off by more than 1/255, PSNR over the whole
panel). The kernel's own error against the FP64 oracle fed the dequantised
attributes is checked by tests/test_gpu_precision.py.
"""
from __future__ import annotations

import argparse
import json
import math


def image_metrics(got, ref):
    """max |err|, share off by > 1/255 and PSNR of clamped images (torch)."""
    g, r = got.clamp(0, 1), ref.clamp(0, 1)
    err = (g - r).abs()
    mse = float((err.double() ** 2).mean())
    return {"max_err": float(err.max()), "frac_off_1_255": float((err > 1 / 255).float().mean()),
            "psnr_db": float("inf") if mse == 0 else 10 * math.log10(1 / mse)}


def run(frames: int = 5, gaussians: int = 0):
    import torch

    from . import lfd, synth

    w = synth.WORKLOADS["precision8k"]
    scene = synth.scene_for(w, gaussians or None)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    # 32x16 tiles at 8K keep the Gaussian-tile pair count below 2^32
    plan = lfd.Plan(w.panel, tile=(32, 16), views_per_cluster=8)
    rows, ref = [], None
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
        if ref is None:
            ref = out.clone()
        row = {"attributes": name, "fps": 1000.0 / ms, "ms_per_frame": ms, "pairs": st["num_pairs"],
               "subpixels_per_s": w.panel.subpixels * 1000.0 / ms,
               "attr_bytes_per_gaussian": 12 + (4 if name == "fp32" else 2) * (3 + 4 + 1 + 48),
               "storage_error_vs_fp32_attributes": image_metrics(out, ref)}
        rows.append(row)
        print(json.dumps(row), flush=True)
        del s, out
    plan.close()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--frames", type=int, default=5)
    ap.add_argument("--gaussians", type=int, default=0)
    args = ap.parse_args()
    run(args.frames, args.gaussians)


if __name__ == "__main__":
    main()
