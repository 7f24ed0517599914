"""Differentiable FP64 restatement of the interlaced render for small scenes.

TEST INFRASTRUCTURE ONLY (imported by the tests): the reference gradient for
the backward pass. Plain PyTorch CPU float64 ops following the same
definitions as the C oracle - Sec. 3.1 Eq. 1-3 (view index, passed in), Eq. 5
(per-view means), Eq. 6 (covariance, depth and SH colour at the cluster's
representative view, Appendix B.1 clusters), Eq. 9-10 with the 3DGS rules -
evaluated by brute force over every Gaussian for every subpixel; autograd
gives the gradient of any loss of the image with respect to the means,
scales, rotations, opacities and SH coefficients.

The discrete decisions (depth order, near-plane culling, the alpha < 1/255
skip, the stop before T < 1e-4, the 0.99 clamp) are taken without gradient,
exactly as the piecewise definition does; the depth order uses the FP32
depth of the Eq. 11 key like the C oracle. Pinned by tests/test_oracle_grad.py
against the C oracle's forward and against central finite differences.
"""
from __future__ import annotations

import math

import numpy as np
import torch

NEAR = 0.2
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def _sh_basis(d: torch.Tensor) -> torch.Tensor:
    """Real SH basis of degree 3 (3DGS convention), d [..., 3] unit -> [..., 16]."""
    pi = math.pi
    c0 = 0.5 * math.sqrt(1.0 / pi)
    c1 = math.sqrt(3.0 / (4.0 * pi))
    c2a, c2b, c2c = 0.5 * math.sqrt(15.0 / pi), 0.25 * math.sqrt(5.0 / pi), 0.25 * math.sqrt(15.0 / pi)
    c3a, c3b = 0.25 * math.sqrt(35.0 / (2.0 * pi)), 0.5 * math.sqrt(105.0 / pi)
    c3c, c3d, c3e = 0.25 * math.sqrt(21.0 / (2.0 * pi)), 0.25 * math.sqrt(7.0 / pi), 0.25 * math.sqrt(105.0 / pi)
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    xx, yy, zz = x * x, y * y, z * z
    return torch.stack([
        torch.full_like(x, c0), -c1 * y, c1 * z, -c1 * x,
        c2a * x * y, -c2a * y * z, c2b * (2 * zz - xx - yy), -c2a * x * z, c2c * (xx - yy),
        -c3a * y * (3 * xx - yy), c3b * x * y * z, -c3c * y * (4 * zz - xx - yy),
        c3d * z * (2 * zz - 3 * xx - 3 * yy), -c3c * x * (4 * zz - xx - yy), c3e * z * (xx - yy),
        -c3a * x * (xx - 3 * yy)], dim=-1)


def _depth_f32(cam: np.ndarray, means32: np.ndarray) -> np.ndarray:
    """((R20 mx + R21 my) + R22 mz) + t2 with float32 rounding at each step."""
    c = cam.astype(np.float32)
    m = means32.astype(np.float32)
    d = (c[6] * m[:, 0]).astype(np.float32) + (c[7] * m[:, 1]).astype(np.float32)
    d = d.astype(np.float32) + (c[8] * m[:, 2]).astype(np.float32)
    return (d.astype(np.float32) + c[11]).astype(np.float32)


def render(params: dict, cams: np.ndarray, V: np.ndarray, c: int, bg=(0.0, 0.0, 0.0),
           alpha_min: float = ALPHA_MIN):
    """params: float64 tensors means [M,3], scales [M,3], quats [M,4] (w,x,y,z),
    opacities [M], sh [M,16,3] (requires_grad as needed). cams float32 [N,16].
    V uint8 [H,W,3]. Returns the image [H,W,3] (float64). alpha_min is the
    skip threshold of Eq. 10 (1/255); the tests move it by +-0.1 % to bracket
    the definition's jump there (the accuracy reading of the render)."""
    means, scales, quats = params["means"], params["scales"], params["quats"]
    opac, sh = params["opacities"], params["sh"]
    H, W, _ = V.shape
    N = cams.shape[0]
    K = (N + c - 1) // c
    M = means.shape[0]
    camt = torch.from_numpy(cams.astype(np.float64))
    means32 = means.detach().numpy().astype(np.float32)

    # per-view means (Eq. 5) and validity
    R = camt[:, :9].reshape(N, 3, 3)
    t = camt[:, 9:12]
    p = torch.einsum("nab,mb->nma", R, means) + t[:, None, :]          # [N, M, 3]
    fx, fy, cx, cy = camt[:, 12], camt[:, 13], camt[:, 14], camt[:, 15]
    mu = torch.stack([fx[:, None] * p[..., 0] / p[..., 2] + cx[:, None],
                      fy[:, None] * p[..., 1] / p[..., 2] + cy[:, None]], dim=-1)  # [N, M, 2]
    vvalid = torch.from_numpy(np.stack([_depth_f32(cams[j], means32) > np.float32(NEAR)
                                        for j in range(N)]))

    # 3D covariance
    q = quats / torch.linalg.norm(quats, dim=1, keepdim=True)
    w_, x_, y_, z_ = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    Rq = torch.stack([
        1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_),
        2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_),
        2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)], dim=1).reshape(M, 3, 3)
    S3 = Rq @ torch.diag_embed(scales * scales) @ Rq.transpose(1, 2)

    out = torch.zeros((H, W, 3), dtype=torch.float64)
    bgv = torch.tensor(bg, dtype=torch.float64)
    xs = torch.arange(W, dtype=torch.float64) + 0.5
    ys = torch.arange(H, dtype=torch.float64) + 0.5
    Vt = torch.from_numpy(V.astype(np.int64))
    for k in range(K):
        jr = min(k * c + c // 2, N - 1)
        cr = cams[jr]
        pr = p[jr]
        zkey = _depth_f32(cr, means32)
        limx = 1.3 * (0.5 * W / float(cr[12]))
        limy = 1.3 * (0.5 * H / float(cr[13]))
        txz = torch.clamp(pr[:, 0] / pr[:, 2], -limx, limx)
        tyz = torch.clamp(pr[:, 1] / pr[:, 2], -limy, limy)
        fxr, fyr = float(cr[12]), float(cr[13])
        zero = torch.zeros_like(txz)
        J = torch.stack([torch.stack([fxr / pr[:, 2], zero, -fxr * txz / pr[:, 2]], dim=1),
                         torch.stack([zero, fyr / pr[:, 2], -fyr * tyz / pr[:, 2]], dim=1)], dim=1)
        Tm = J @ R[jr]                                                   # [M, 2, 3]
        S2 = Tm @ S3 @ Tm.transpose(1, 2) + 0.3 * torch.eye(2, dtype=torch.float64)
        det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
        ca, cb, cc = S2[:, 1, 1] / det, -S2[:, 0, 1] / det, S2[:, 0, 0] / det
        cpos = -(R[jr].T @ t[jr])
        d = means - cpos[None, :]
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        col = torch.clamp(torch.einsum("mc,mcu->mu", _sh_basis(d), sh) + 0.5, min=0.0)
        valid = (zkey > np.float32(NEAR)) & (det.detach().numpy() > 0) & (opac.detach().numpy() >= alpha_min)
        idx = np.nonzero(valid)[0]
        idx = idx[np.lexsort((idx, zkey[idx].astype(np.float64)))]
        if len(idx) == 0:
            sel = (Vt // c) == k
            out = torch.where(sel, bgv.expand(H, W, 3), out)
            continue
        it = torch.from_numpy(idx)
        for j in range(k * c, min(k * c + c, N)):
            sel = Vt == j                                                # [H, W, 3]
            if not bool(sel.any()):
                continue
            m2 = mu[j][it]                                               # [G, 2]
            dx = xs[None, :, None] - m2[None, None, :, 0]                # [1, W, G]
            dy = ys[:, None, None] - m2[None, None, :, 1]                # [H, 1, G]
            qf = ca[it] * dx * dx + 2 * cb[it] * dx * dy + cc[it] * dy * dy  # [H, W, G]
            power = -0.5 * qf
            v = opac[it] * torch.exp(power)
            keep = (power <= 0) & (v >= alpha_min) & vvalid[j][it][None, None, :]
            alpha = torch.where(keep, torch.minimum(v, torch.full_like(v, ALPHA_MAX)), torch.zeros_like(v))
            one_minus = 1 - alpha
            T_after = torch.cumprod(one_minus, dim=-1)
            T_before = torch.cat([torch.ones_like(T_after[..., :1]), T_after[..., :-1]], dim=-1)
            stop = ((T_after < T_MIN) & keep).detach()
            first = torch.where(stop.any(-1), stop.float().argmax(-1), torch.full(stop.shape[:-1], stop.shape[-1]))
            live = torch.arange(alpha.shape[-1])[None, None, :] < first[..., None]
            wgt = torch.where(live, alpha * T_before, torch.zeros_like(alpha))
            # transmittance after the last added Gaussian
            n_add = live.sum(-1)
            T_fin = torch.where(n_add > 0, torch.gather(T_after, -1, (n_add - 1).clamp(min=0)[..., None])[..., 0],
                                torch.ones_like(n_add, dtype=torch.float64))
            img = torch.einsum("hwg,gu->hwu", wgt, col[it]) + T_fin[..., None] * bgv
            out = torch.where(sel, img, out)
    return out
