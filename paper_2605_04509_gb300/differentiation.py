"""Optimisation steps through the differentiable interlaced render (the
differentiation workload): 500k Gaussians, 24 views, a
1920x1080 panel (slant 0.2 rad, pitch 4.8 subpixels), clusters of 8 views,
L2 loss to a target interlaced image rendered from a copy whose means are
perturbed by N(0, 0.01) (seed 6).

    python -m paper_2605_04509_gb300.differentiation [--steps 10]

Each step is forward (lfd_render, keeping each subpixel's final
transmittance and stop position) + loss + backward (lfd_render_backward: each
(tile, cluster) run walked back to front from the kept state, then the 3DGS
projection chain) through lfd.render_autograd, then one plain gradient step
on the means. Prints steps/s, the forward and backward times, the loss
before and after, and the gradient norms per parameter group; then the same
for the backward that re-blends each list first (nothing kept by the
forward), under "replay". The gradients
themselves are checked against the FP64 autograd oracle (itself pinned to
finite differences) by tests/test_gpu_backward.py.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def run(steps: int = 10, lr: float = 1e-4):
    import torch

    from . import lfd, synth

    w = synth.WORKLOADS["diff1080"]
    scene = synth.scene_for(w)
    cams = synth.arc_cameras(w.rig, w.panel.width, w.panel.height)
    rng = np.random.default_rng(6)
    moved = dict(scene)
    moved["means"] = (scene["means"] + rng.normal(0, 0.01, scene["means"].shape)).astype(np.float32)
    plan = lfd.Plan(w.panel, views_per_cluster=8)
    target, _ = plan.render(lfd.scene_to_device(moved), cams)
    target = target.clone()
    keys = ("means", "scales", "quats", "opacities", "sh")

    def optimise(keep_state: bool):
        """`steps` timed optimisation steps from the unperturbed scene."""
        leaves = {k: v.clone().requires_grad_(True) for k, v in lfd.scene_to_device(scene).items()}

        def step(apply: bool):
            for v in leaves.values():
                v.grad = None
            img = lfd.render_autograd(plan, cams, *(leaves[k] for k in keys), keep_state=keep_state)
            loss = ((img - target) ** 2).sum()
            loss.backward()
            if apply:
                with torch.no_grad():
                    leaves["means"] -= lr * leaves["means"].grad
            return loss

        loss0 = float(step(False).detach())
        for _ in range(2):
            step(False)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        for _ in range(steps):
            loss = step(True)
        e[1].record()
        torch.cuda.synchronize()
        ms_step = e[0].elapsed_time(e[1]) / steps
        # forward alone (same flags), for the split
        f = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.no_grad():
            scene_now = {k: v.detach() for k, v in leaves.items()}
            f[0].record()
            for _ in range(steps):
                plan.render(scene_now, cams)
            f[1].record()
        torch.cuda.synchronize()
        ms_fwd = f[0].elapsed_time(f[1]) / steps
        return {"ms_per_step": ms_step, "steps_per_s": 1000.0 / ms_step, "ms_forward": ms_fwd,
                "ms_backward_and_loss": ms_step - ms_fwd, "loss_first": loss0,
                "loss_last": float(loss.detach()),
                "grad_norms": {k: float(leaves[k].grad.norm()) for k in keys}}

    kept = optimise(True)
    replay = optimise(False)
    line = {
        "workload": "diff1080: 500k Gaussians, 24 views, 1920x1080 panel, |V_k| = 8, L2 loss to a "
                    "target rendered from means + N(0, 0.01)",
        "steps": steps,
        **kept,
        "replay": {k: replay[k] for k in ("ms_per_step", "steps_per_s", "ms_forward",
                                          "ms_backward_and_loss", "loss_last")},
        "replay_note": "backward re-blends each (tile, cluster) list to find each subpixel's final "
                       "transmittance instead of reading the 8 bytes per subpixel the forward kept",
    }
    print(json.dumps(line), flush=True)
    plan.close()
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    run(args.steps)


if __name__ == "__main__":
    main()
