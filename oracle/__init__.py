"""FP64 CPU oracle for subpixel-level 3DGS light-field rasterisation.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. It is a plain, slow
restatement of the paper's definitions (Sec. 3.1 Eq. 1-3, Sec. 4.1-4.3
Eq. 4-10, Appendix B) in C, loaded through ctypes, and shares no code with
the CUDA library.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the image-quality effect of attribute reuse for clusters of more than one
view (Eq. 6), which is "parity unpinned" against the paper's trained-scene
numbers; it is pinned only through the one-view-per-cluster identity.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfd_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblfd_oracle.so")
_lib = None

ALPHA_MIN = 1.0 / 255.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lfd_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
            "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ct.CDLL(_LIB)
        _declare(_lib)
    return _lib


_P = ct.c_void_p
_I = ct.c_int
_L = ct.c_int64
_D = ct.c_double


def _declare(L):
    sig = {
        "orc_view_index": [_I, _I, _I, _D, _D, _D, _P],
        "orc_remap": [_I, _I, _I, _P, _I, _I, _I, _P, _P, _P],
        "orc_clusters": [_I, _I, _P, _P],
        "orc_project": [_L, _P, _P, _P, _P, _P, _I, _I, _P, _I, _I, _I,
                        _P, _P, _P, _P, _P, _P, _P],
        "orc_render": [_I, _I, _I, _I, _P, _I, _I, _L, _P, _P, _P, _P, _P, _P, _P,
                       _I, _I, _I, _I, _I, _P, _P, _P],
        "orc_blend_lists": [_I, _I, _I, _I, _P, _I, _I, _L, _P, _P, _P, _P, _P,
                            _P, _P, _I, _I, _I, _I, _P, _P, _P],
        "orc_render_fullframe": [_I, _I, _I, _P, _L, _P, _P, _P, _P, _P, _P, _P,
                                 _I, _I, _I, _I, _P, _P],
        "orc_mirror_count": [_I, _I, _I, _I, _I, _I, _L, _P, _P, _P, _P],
        "orc_mirror_emit": [_I, _I, _I, _I, _I, _I, _L, _P, _P, _P, _P, _P, _P, _P],
        "orc_mirror_sort": [_L, _P, _P],
        "orc_mirror_ranges": [_L, _P, _I, _I, _I, _P],
        "orc_num_threads": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _I
    L.orc_set_alpha_min.argtypes = [_D]
    L.orc_set_alpha_min.restype = _D


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ct.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return lib().orc_num_threads()


class alpha_min:
    """Context manager rendering with a different alpha skip threshold."""

    def __init__(self, value: float):
        self.value = value
        self.old = None

    def __enter__(self):
        self.old = lib().orc_set_alpha_min(float(self.value))
        return self

    def __exit__(self, *exc):
        lib().orc_set_alpha_min(self.old)
        return False


def render_bracket(proj, V, c, crop=None, rel: float = 1e-3, **kw):
    """The definition rendered at the 1/255 threshold and at (1 -/+ rel) of it;
    returns (image, lower-threshold image, upper-threshold image)."""
    ref, _ = render(proj, V, c, crop=crop, **kw)
    with alpha_min(ALPHA_MIN * (1 - rel)):
        lo, _ = render(proj, V, c, crop=crop, **kw)
    with alpha_min(ALPHA_MIN * (1 + rel)):
        hi, _ = render(proj, V, c, crop=crop, **kw)
    return ref, lo, hi


def num_clusters(n: int, c: int) -> int:
    return (n + c - 1) // c


def view_index(panel) -> np.ndarray:
    """Eq. 1-3: uint8 [H, W, 3]."""
    V = np.zeros((panel.height, panel.width, 3), dtype=np.uint8)
    _check(lib().orc_view_index(panel.width, panel.height, panel.num_views,
                                float(panel.tan_slant), float(panel.pitch),
                                float(panel.k_offset), _ptr(V)), "view_index")
    return V


def remap(V: np.ndarray, num_views: int, tile_w: int, tile_h: int, c: int):
    """Sec. 4.3: (psi [T, TW*TH*3] uint16, n_sub [T], seg [T, K+1])."""
    H, W, _ = V.shape
    T = ((W + tile_w - 1) // tile_w) * ((H + tile_h - 1) // tile_h)
    K = num_clusters(num_views, c)
    psi = np.zeros((T, tile_w * tile_h * 3), dtype=np.uint16)
    n_sub = np.zeros(T, dtype=np.int32)
    seg = np.zeros((T, K + 1), dtype=np.int32)
    _check(lib().orc_remap(W, H, num_views, _ptr(np.ascontiguousarray(V)), tile_w, tile_h, c,
                           _ptr(psi), _ptr(n_sub), _ptr(seg)), "remap")
    return psi, n_sub, seg


def clusters(n: int, c: int) -> Tuple[np.ndarray, np.ndarray]:
    """Appendix B.1: (slot_view [K, C], representative view [K])."""
    K = num_clusters(n, c)
    slot = np.zeros((K, c), dtype=np.int32)
    rep = np.zeros(K, dtype=np.int32)
    _check(lib().orc_clusters(n, c, _ptr(slot), _ptr(rep)), "clusters")
    return slot, rep


def project(scene: Dict[str, np.ndarray], cams: np.ndarray, width: int, height: int,
            c: int, sh_degree: int = 3) -> Dict[str, np.ndarray]:
    """Eq. 4-6 in FP64. Per view: mean2d [N, M, 2], vvalid [N, M]; per cluster:
    conic [K, M, 3], depth [K, M], color [K, M, 3], tau [K, M], valid [K, M]."""
    means = np.ascontiguousarray(scene["means"], dtype=np.float32)
    M = means.shape[0]
    N = cams.shape[0]
    K = num_clusters(N, c)
    ncoef = (sh_degree + 1) ** 2
    sh = np.ascontiguousarray(scene["sh"][:, :ncoef, :], dtype=np.float32)
    out = {
        "mean2d": np.zeros((N, M, 2)), "vvalid": np.zeros((N, M), dtype=np.uint8),
        "conic": np.zeros((K, M, 3)), "depth": np.zeros((K, M)),
        "color": np.zeros((K, M, 3)), "tau": np.zeros((K, M)),
        "valid": np.zeros((K, M), dtype=np.uint8),
    }
    _check(lib().orc_project(
        M, _ptr(means), _ptr(np.ascontiguousarray(scene["scales"], dtype=np.float32)),
        _ptr(np.ascontiguousarray(scene["quats"], dtype=np.float32)),
        _ptr(np.ascontiguousarray(scene["opacities"], dtype=np.float32)), _ptr(sh), sh_degree,
        N, _ptr(np.ascontiguousarray(cams, dtype=np.float32)), width, height, c,
        _ptr(out["mean2d"]), _ptr(out["vvalid"]), _ptr(out["conic"]), _ptr(out["depth"]),
        _ptr(out["color"]), _ptr(out["tau"]), _ptr(out["valid"])), "project")
    out["opac"] = np.ascontiguousarray(scene["opacities"], dtype=np.float64)
    return out


def render(proj: Dict[str, np.ndarray], V: np.ndarray, c: int, crop=None, mode: int = 1,
           tile: Tuple[int, int] = (16, 16), bg=(0.0, 0.0, 0.0)) -> Tuple[np.ndarray, int]:
    """Eq. 9-10 per subpixel of the crop (x0, y0, x1, y1). Returns
    (image [y1-y0, x1-x0, 3] float64, visited list entries)."""
    H, W, _ = V.shape
    N = proj["mean2d"].shape[0]
    M = proj["mean2d"].shape[1]
    x0, y0, x1, y1 = crop if crop is not None else (0, 0, W, H)
    out = np.zeros((y1 - y0, x1 - x0, 3))
    n = ct.c_int64(0)
    bgv = np.asarray(bg, dtype=np.float64)
    _check(lib().orc_render(
        W, H, N, c, _ptr(np.ascontiguousarray(V)), tile[0], tile[1], M,
        _ptr(proj["mean2d"]), _ptr(proj["vvalid"]), _ptr(proj["conic"]), _ptr(proj["depth"]),
        _ptr(proj["color"]), _ptr(proj["valid"]), _ptr(proj["opac"]),
        x0, y0, x1, y1, mode, _ptr(bgv), _ptr(out), ct.byref(n)), "render")
    return out, n.value


def blend_lists(proj: Dict[str, np.ndarray], V: np.ndarray, c: int, ranges: np.ndarray,
                lst: np.ndarray, crop=None, tile=(16, 16), bg=(0.0, 0.0, 0.0)):
    """Eq. 9-10 along given (tile, cluster) lists. ranges: uint32 [T, K, 2]."""
    H, W, _ = V.shape
    N, M = proj["mean2d"].shape[:2]
    x0, y0, x1, y1 = crop if crop is not None else (0, 0, W, H)
    out = np.zeros((y1 - y0, x1 - x0, 3))
    n = ct.c_int64(0)
    bgv = np.asarray(bg, dtype=np.float64)
    lst = np.ascontiguousarray(lst, dtype=np.uint32)
    if lst.size == 0:
        lst = np.zeros(1, dtype=np.uint32)
    _check(lib().orc_blend_lists(
        W, H, N, c, _ptr(np.ascontiguousarray(V)), tile[0], tile[1], M,
        _ptr(proj["mean2d"]), _ptr(proj["vvalid"]), _ptr(proj["conic"]), _ptr(proj["color"]),
        _ptr(proj["opac"]), _ptr(np.ascontiguousarray(ranges, dtype=np.uint32)), _ptr(lst),
        x0, y0, x1, y1, _ptr(bgv), _ptr(out), ct.byref(n)), "blend_lists")
    return out, n.value


def render_fullframe(proj1: Dict[str, np.ndarray], V: np.ndarray, crop=None,
                     bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Every view rendered as a full 3DGS image, then interlaced by V.
    ``proj1`` must be a projection with one view per cluster."""
    H, W, _ = V.shape
    N, M = proj1["mean2d"].shape[:2]
    assert proj1["conic"].shape[0] == N, "full-frame rendering needs per-view attributes"
    x0, y0, x1, y1 = crop if crop is not None else (0, 0, W, H)
    out = np.zeros((y1 - y0, x1 - x0, 3))
    bgv = np.asarray(bg, dtype=np.float64)
    _check(lib().orc_render_fullframe(
        W, H, N, _ptr(np.ascontiguousarray(V)), M, _ptr(proj1["mean2d"]),
        _ptr(proj1["vvalid"]), _ptr(proj1["conic"]), _ptr(proj1["depth"]),
        _ptr(proj1["color"]), _ptr(proj1["valid"]), _ptr(proj1["opac"]),
        x0, y0, x1, y1, _ptr(bgv), _ptr(out)), "render_fullframe")
    return out


# ---------------------------------------------------------------------------
# FP32 mirror: tile bins, Eq. 11 keys, sorted list and range table.
# ---------------------------------------------------------------------------

def ceil_log2(v: int) -> int:
    b = 0
    while (1 << b) < v:
        b += 1
    return b


def mirror_count(width, height, tile, conic, tau, means_kc) -> np.ndarray:
    """Tile count of the cluster union per (k, i). conic f32 [K, M, 3],
    tau f32 [K, M], means_kc f32 [K, M, C, 2]."""
    K, M, C, _ = means_kc.shape
    counts = np.zeros((K, M), dtype=np.uint32)
    _check(lib().orc_mirror_count(
        width, height, tile[0], tile[1], K, C, M,
        _ptr(np.ascontiguousarray(conic, dtype=np.float32)),
        _ptr(np.ascontiguousarray(tau, dtype=np.float32)),
        _ptr(np.ascontiguousarray(means_kc, dtype=np.float32)), _ptr(counts)), "mirror_count")
    return counts


def mirror_keys(width, height, tile, conic, tau, depth, means_kc):
    """Eq. 11 keys and Gaussian ids in (k, i) emission order."""
    K, M, C, _ = means_kc.shape
    counts = mirror_count(width, height, tile, conic, tau, means_kc)
    flat = counts.reshape(-1).astype(np.uint64)
    offsets = np.zeros_like(flat)
    if flat.size:
        offsets[1:] = np.cumsum(flat)[:-1]
    P = int(flat.sum())
    keys = np.zeros(max(P, 1), dtype=np.uint64)
    vals = np.zeros(max(P, 1), dtype=np.uint32)
    _check(lib().orc_mirror_emit(
        width, height, tile[0], tile[1], K, C, M,
        _ptr(np.ascontiguousarray(conic, dtype=np.float32)),
        _ptr(np.ascontiguousarray(tau, dtype=np.float32)),
        _ptr(np.ascontiguousarray(depth, dtype=np.float32)),
        _ptr(np.ascontiguousarray(means_kc, dtype=np.float32)),
        _ptr(offsets), _ptr(keys), _ptr(vals)), "mirror_emit")
    return counts, keys[:P], vals[:P]


def mirror_sort(keys: np.ndarray, vals: np.ndarray):
    k = np.array(keys, dtype=np.uint64, copy=True)
    v = np.array(vals, dtype=np.uint32, copy=True)
    if k.size:
        _check(lib().orc_mirror_sort(k.size, _ptr(k), _ptr(v)), "mirror_sort")
    return k, v


def mirror_ranges(keys_sorted: np.ndarray, num_tiles: int, K: int) -> np.ndarray:
    ranges = np.zeros((num_tiles, K, 2), dtype=np.uint32)
    ks = np.ascontiguousarray(keys_sorted, dtype=np.uint64)
    if ks.size == 0:
        ks = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_mirror_ranges(keys_sorted.size, _ptr(ks), ceil_log2(K), num_tiles, K,
                                   _ptr(ranges)), "mirror_ranges")
    return ranges


def mirror_lists(width, height, tile, conic, tau, depth, means_kc):
    """Full FP32 mirror of key generation, sort and range identification:
    returns dict(counts, keys, vals (emission order), keys_sorted, list, ranges)."""
    K = means_kc.shape[0]
    T = ((width + tile[0] - 1) // tile[0]) * ((height + tile[1] - 1) // tile[1])
    counts, keys, vals = mirror_keys(width, height, tile, conic, tau, depth, means_kc)
    ks, vs = mirror_sort(keys, vals)
    ranges = mirror_ranges(ks, T, K)
    return {"counts": counts, "keys": keys, "vals": vals, "keys_sorted": ks, "list": vs,
            "ranges": ranges}


def means_by_slot(mean2d: np.ndarray, vvalid: np.ndarray, c: int) -> np.ndarray:
    """Per-view means [N, M, 2] -> cluster-slot layout [K, M, C, 2] (float64),
    with NaN where the Gaussian is culled in that view."""
    N, M, _ = mean2d.shape
    slot, _rep = clusters(N, c)
    m = np.where(vvalid[..., None].astype(bool), mean2d, np.nan)
    return np.ascontiguousarray(np.transpose(m[slot], (0, 2, 1, 3)))


def per_view_from_slots(means_kc: np.ndarray, num_views: int, c: int):
    """Cluster-slot means [K, M, C, 2] -> per-view means [N, M, 2] (float64)
    and validity [N, M] (finite means)."""
    K, M, C, _ = means_kc.shape
    out = np.zeros((num_views, M, 2))
    for j in range(num_views):
        out[j] = means_kc[j // c, :, j % c, :]
    vvalid = np.isfinite(out).all(axis=2).astype(np.uint8)
    out = np.where(vvalid[..., None].astype(bool), out, 0.0)
    return np.ascontiguousarray(out), np.ascontiguousarray(vvalid)
