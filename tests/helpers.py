"""Shared test helpers: image error metrics and workload construction."""
import math

import numpy as np

MAX_ERR = 2e-3          # max |err| per subpixel, values clamped to [0, 1]
MAX_FRAC_OFF = 1e-3     # fraction of subpixels off by more than 1/255


def image_metrics(got, ref):
    """Error of a render against the FP64 oracle on clamped [0, 1] values."""
    g = np.clip(np.asarray(got, np.float64), 0.0, 1.0)
    r = np.clip(np.asarray(ref, np.float64), 0.0, 1.0)
    err = np.abs(g - r)
    mse = float((err ** 2).mean()) if err.size else 0.0
    return {
        "max_err": float(err.max()) if err.size else 0.0,
        "frac_off": float((err > 1.0 / 255.0).mean()) if err.size else 0.0,
        "psnr": float("inf") if mse == 0 else 10 * math.log10(1.0 / mse),
    }


def assert_image_close(got, ref, what=""):
    m = image_metrics(got, ref)
    assert m["max_err"] <= MAX_ERR and m["frac_off"] <= MAX_FRAC_OFF, f"{what}: {m}"
    return m


THRESHOLD_REL = 1e-3  # relative move of the 1/255 skip threshold that brackets the definition


def assert_render_matches(got, ref, lo, hi, what=""):
    """Tolerance check against the FP64 definition, aware of its discontinuity
    at alpha = 1/255. ``lo``/``hi`` are the definition rendered with the skip
    threshold moved by -/+0.1 %. Where those differ from ``ref`` by more than
    half the tolerance the definition itself jumps (a Gaussian's ~1/255
    contribution appears or not), so the render must lie within that spread
    (+ the tolerance); everywhere else the plain bar applies: max |err| <= 2e-3.
    At most 0.1 % of subpixels may be off by more than 1/255 in all cases."""
    g = np.clip(np.asarray(got, np.float64), 0.0, 1.0)
    r = np.clip(np.asarray(ref, np.float64), 0.0, 1.0)
    a = np.clip(np.asarray(lo, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(hi, np.float64), 0.0, 1.0)
    low = np.minimum(np.minimum(r, a), b)
    high = np.maximum(np.maximum(r, a), b)
    jump = (high - low) > MAX_ERR / 2
    err = np.abs(g - r)
    m = image_metrics(got, ref)
    m["max_err_regular"] = float(err[~jump].max()) if (~jump).any() else 0.0
    m["threshold_jumps"] = int(jump.sum())
    outside = (g < low - MAX_ERR) | (g > high + MAX_ERR)
    assert m["max_err_regular"] <= MAX_ERR, f"{what}: {m}"
    assert not outside.any(), f"{what}: {int(outside.sum())} outside the bracket: {m}"
    assert m["frac_off"] <= MAX_FRAC_OFF, f"{what}: {m}"
    return m
