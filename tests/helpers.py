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
