"""Thin ctypes binding of liblfd.so (include/lfd.h).

Argument marshalling only: every step of the renderer runs in the library's
CUDA kernels. PyTorch supplies device memory and streams. If the library has
not been built, every entry point raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblfd.so")

LFD_OK = 0
LFD_ERR_INVALID = -1
LFD_ERR_OOM = -2
LFD_ERR_CAPACITY = -3
LFD_ERR_CUDA = -4
LFD_ERR_STATE = -5
LFD_ERR_TIMEOUT = -6
SORT_DEPTH_FIRST = 0
SORT_KEY64 = 1
FLAG_STAGE_TIMING = 1
FLAG_COUNT_EVALS = 2
FLAG_KEEP_BLEND_STATE = 4


class LFDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lfd status {status}: {message}")
        self.status = status


class CPanel(ct.Structure):
    _fields_ = [("width", ct.c_int32), ("height", ct.c_int32), ("num_views", ct.c_int32),
                ("tan_slant", ct.c_double), ("pitch", ct.c_double), ("k_offset", ct.c_double)]


class COpts(ct.Structure):
    _fields_ = [("tile_w", ct.c_int32), ("tile_h", ct.c_int32),
                ("views_per_cluster", ct.c_int32), ("remap", ct.c_int32),
                ("sort_mode", ct.c_int32), ("bg", ct.c_float * 3),
                ("subpixels_per_thread", ct.c_int32)]


DTYPE_F32 = 0
DTYPE_F16 = 1
DTYPE_BF16 = 2


class CGaussians(ct.Structure):
    _fields_ = [("means", ct.c_void_p), ("scales", ct.c_void_p), ("quats", ct.c_void_p),
                ("opacities", ct.c_void_p), ("sh", ct.c_void_p), ("count", ct.c_int64),
                ("sh_degree", ct.c_int32), ("attr_dtype", ct.c_int32)]


class CCamera(ct.Structure):
    _fields_ = [("v", ct.c_float * 16)]


class CPlanInfo(ct.Structure):
    _fields_ = [("num_clusters", ct.c_int32), ("tiles_x", ct.c_int32), ("tiles_y", ct.c_int32),
                ("tile_capacity", ct.c_int32), ("bit_k", ct.c_int32), ("bit_t", ct.c_int32),
                ("max_segment", ct.c_int32)]


class CStats(ct.Structure):
    _fields_ = [("num_pairs", ct.c_int64), ("num_visits", ct.c_int64), ("num_evals", ct.c_int64),
                ("ms_project", ct.c_float), ("ms_keygen", ct.c_float),
                ("ms_sort", ct.c_float), ("ms_blend", ct.c_float)]

    def as_dict(self) -> Dict[str, float]:
        return {f: getattr(self, f) for f, _ in self._fields_}


class CStageTotals(ct.Structure):
    _fields_ = [("frames", ct.c_int64), ("ms_project", ct.c_double), ("ms_keygen", ct.c_double),
                ("ms_sort", ct.c_double), ("ms_blend", ct.c_double)]


_lib = None
_P = ct.c_void_p


def load() -> ct.CDLL:
    """Load liblfd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LFDError(LFD_ERR_STATE, f"{LIB_PATH} is missing: build it with "
                           "paper_2605_04509_gb300.build_lib.build()")
        L = ct.CDLL(LIB_PATH)
        sig = {
            "lfd_plan_create": ([ct.POINTER(CPanel), ct.POINTER(COpts), ct.POINTER(_P)], ct.c_int),
            "lfd_plan_destroy": ([_P], None),
            "lfd_plan_get_info": ([_P, ct.POINTER(CPlanInfo)], ct.c_int),
            "lfd_set_flags": ([_P, ct.c_int32], ct.c_int),
            "lfd_plan_copy_tables": ([_P, _P, _P, _P, _P], ct.c_int),
            "lfd_project": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32,
                             _P, _P, _P, _P, _P], ct.c_int),
            "lfd_render_projected": ([_P, ct.c_int64, _P, _P, _P, _P, _P, _P,
                                      ct.POINTER(CStats)], ct.c_int),
            "lfd_render": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32, _P, _P,
                            ct.POINTER(CStats)], ct.c_int),
            "lfd_render_projected_noalloc": ([_P, ct.c_int64, _P, _P, _P, _P, _P, _P,
                                              ct.POINTER(CStats)], ct.c_int),
            "lfd_render_host_async": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32,
                                       _P, _P, ct.POINTER(CStats)], ct.c_int),
            "lfd_render_host_wait": ([_P], ct.c_int),
            "lfd_render_host": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32,
                                 _P, _P, ct.POINTER(CStats)], ct.c_int),
            "lfd_render_backward": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32,
                                     _P, _P, _P, _P, _P, _P, _P], ct.c_int),
            "lfd_render_fullframe": ([_P, ct.POINTER(CGaussians), ct.POINTER(CCamera), ct.c_int32,
                                      _P, _P, ct.POINTER(CStats)], ct.c_int),
            "lfd_plan_copy_lists": ([_P, _P, _P, _P, ct.c_int64], ct.c_int),
            "lfd_get_stage_totals": ([_P, ct.POINTER(CStageTotals), ct.c_int32], ct.c_int),
            "lfd_plan_reserve": ([_P, ct.c_int64, ct.c_int64], ct.c_int),
            "lfd_plan_status": ([_P, ct.POINTER(ct.c_int64)], ct.c_int),
            "lfd_batch_create": ([ct.POINTER(_P), ct.c_int32, ct.POINTER(_P)], ct.c_int),
            "lfd_batch_destroy": ([_P], None),
            "lfd_batch_reserve": ([_P, ct.POINTER(ct.c_int64), ct.c_int64], ct.c_int),
            "lfd_batch_render": ([_P, _P, _P, _P, _P], ct.c_int),
            "lfd_batch_status": ([_P, ct.POINTER(ct.c_int64)], ct.c_int),
            "lfd_selftest_wait_timeout": ([_P], ct.c_int),
            "lfd_measure_alu_peaks": ([ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), _P], ct.c_int),
            "lfd_kernel_launches": ([], ct.c_uint64),
            "lfd_make_arc_cameras": ([ct.c_int32, ct.c_double, ct.c_double, ct.c_double, ct.c_int32,
                                      ct.c_int32, ct.POINTER(CCamera)], ct.c_int),
            "lfd_status_string": ([ct.c_int], ct.c_char_p),
            "lfd_last_error": ([], ct.c_char_p),
            "lfd_version": ([], ct.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != LFD_OK:
        L = load()
        raise LFDError(rc, f"{L.lfd_status_string(rc).decode()}: {L.lfd_last_error().decode()}")


def _dptr(t) -> int:
    """Device pointer of a torch CUDA tensor (or 0 for None)."""
    if t is None:
        return 0
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def cameras_array(cams: np.ndarray):
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    arr = (CCamera * len(cams))()
    ct.memmove(arr, cams.ctypes.data, cams.nbytes)
    return arr, len(cams)


def num_sh_degree(sh_shape) -> int:
    ncoef = sh_shape[1]
    return {1: 0, 4: 1, 9: 2, 16: 3}[ncoef]


def gaussians_struct(scene, host: bool = False) -> CGaussians:
    """scene: dict of contiguous float32 tensors means [M,3], scales [M,3],
    quats [M,4], opacities [M], sh [M,(d+1)^2,3] (CUDA, or CPU for host=True)."""
    g = CGaussians()
    ptr = (lambda t: t.data_ptr()) if host else _dptr
    g.means = ptr(scene["means"])
    g.scales = ptr(scene["scales"])
    g.quats = ptr(scene["quats"])
    g.opacities = ptr(scene["opacities"])
    g.sh = ptr(scene["sh"])
    g.count = int(scene["means"].shape[0])
    g.sh_degree = num_sh_degree(tuple(scene["sh"].shape))
    g.attr_dtype = _attr_dtype(scene["scales"])
    for key in ("quats", "opacities", "sh"):
        assert _attr_dtype(scene[key]) == g.attr_dtype, "attributes must share one storage type"
    return g


def _attr_dtype(t) -> int:
    name = str(t.dtype).split(".")[-1]
    kinds = {"float32": DTYPE_F32, "float16": DTYPE_F16, "bfloat16": DTYPE_BF16}
    if name not in kinds:
        raise TypeError(f"unsupported attribute dtype {t.dtype}")
    return kinds[name]


class Plan:
    """A panel + options plan (lfd_plan_create); owns V, Psi and scratch."""

    def __init__(self, panel, tile: Tuple[int, int] = (16, 16), views_per_cluster: int = 8,
                 sort_mode: int = SORT_DEPTH_FIRST, bg=(0.0, 0.0, 0.0), remap: bool = True,
                 subpixels_per_thread: int = 0):
        L = load()
        self.panel = panel
        cp = CPanel(panel.width, panel.height, panel.num_views, float(panel.tan_slant),
                    float(panel.pitch), float(panel.k_offset))
        co = COpts(tile[0], tile[1], views_per_cluster, 1 if remap else 0, sort_mode,
                   (ct.c_float * 3)(*bg), subpixels_per_thread)
        self.subpixels_per_thread = subpixels_per_thread
        h = _P()
        _check(L.lfd_plan_create(ct.byref(cp), ct.byref(co), ct.byref(h)))
        self._h = h
        self.flags = 0
        self._pending = []  # host tensors of queued lfd_render_host_async frames
        self.tile = tuple(tile)
        self.views_per_cluster = views_per_cluster
        self.sort_mode = sort_mode
        info = CPlanInfo()
        _check(L.lfd_plan_get_info(h, ct.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in info._fields_}
        self.K = self.info["num_clusters"]
        self.T = self.info["tiles_x"] * self.info["tiles_y"]

    def close(self):
        if getattr(self, "_h", None):
            load().lfd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_flags(self, flags: int):
        _check(load().lfd_set_flags(self._h, flags))
        self.flags = flags

    def tables(self):
        p = self.panel
        V = np.zeros((p.height, p.width, 3), np.uint8)
        cap = self.info["tile_capacity"]
        psi = np.zeros((self.T, cap), np.uint16)
        n_sub = np.zeros(self.T, np.int32)
        seg = np.zeros((self.T, self.K + 1), np.int32)
        _check(load().lfd_plan_copy_tables(self._h, V.ctypes.data, psi.ctypes.data,
                                           n_sub.ctypes.data, seg.ctypes.data))
        return V, psi, n_sub, seg

    def alloc_projected(self, M: int):
        import torch
        C, K = self.views_per_cluster, self.K
        dev = torch.device("cuda")
        return {
            "means2d": torch.empty((K, M, C, 2), dtype=torch.float32, device=dev),
            "conic_opacity": torch.empty((K, M, 4), dtype=torch.float32, device=dev),
            "color_tau": torch.empty((K, M, 4), dtype=torch.float32, device=dev),
            "depth": torch.empty((K, M), dtype=torch.float32, device=dev),
        }

    def project(self, scene, cams: np.ndarray, out=None, stream=None):
        M = int(scene["means"].shape[0])
        out = out if out is not None else self.alloc_projected(M)
        g = gaussians_struct(scene)
        carr, n = cameras_array(cams)
        _check(load().lfd_project(self._h, ct.byref(g), carr, n, _dptr(out["means2d"]),
                                  _dptr(out["conic_opacity"]), _dptr(out["color_tau"]),
                                  _dptr(out["depth"]), _stream_ptr(stream)))
        return out

    def _image(self, out):
        import torch
        if out is None:
            p = self.panel
            out = torch.empty((p.height, p.width, 3), dtype=torch.float32, device="cuda")
        return out

    def render_projected(self, attrs, out=None, stream=None) -> Tuple[object, Dict]:
        M = int(attrs["depth"].shape[1])
        out = self._image(out)
        st = CStats()
        _check(load().lfd_render_projected(
            self._h, M, _dptr(attrs["means2d"]), _dptr(attrs["conic_opacity"]),
            _dptr(attrs["color_tau"]), _dptr(attrs["depth"]), _dptr(out),
            _stream_ptr(stream), ct.byref(st)))
        return out, st.as_dict()

    def render_projected_noalloc(self, attrs, out=None, stream=None) -> Tuple[object, Dict]:
        """lfd_render_projected_noalloc: the same stages with the library's
        fixed scratch array (small frames only; no device allocation)."""
        M = int(attrs["depth"].shape[1])
        out = self._image(out)
        st = CStats()
        _check(load().lfd_render_projected_noalloc(
            self._h, M, _dptr(attrs["means2d"]), _dptr(attrs["conic_opacity"]),
            _dptr(attrs["color_tau"]), _dptr(attrs["depth"]), _dptr(out),
            _stream_ptr(stream), ct.byref(st)))
        return out, st.as_dict()

    def render(self, scene, cams: np.ndarray, out=None, stream=None) -> Tuple[object, Dict]:
        out = self._image(out)
        g = gaussians_struct(scene)
        carr, n = cameras_array(cams)
        st = CStats()
        _check(load().lfd_render(self._h, ct.byref(g), carr, n, _dptr(out), _stream_ptr(stream),
                                 ct.byref(st)))
        return out, st.as_dict()

    def backward(self, scene, cams: np.ndarray, grad_rgb, stream=None) -> Dict[str, object]:
        """lfd_render_backward for the plan's last render(scene, cams)."""
        import torch
        grads = {k: torch.empty_like(scene[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
        g = gaussians_struct(scene)
        carr, n = cameras_array(cams)
        _check(load().lfd_render_backward(
            self._h, ct.byref(g), carr, n, _dptr(grad_rgb.contiguous()), _dptr(grads["means"]),
            _dptr(grads["scales"]), _dptr(grads["quats"]), _dptr(grads["opacities"]),
            _dptr(grads["sh"]), _stream_ptr(stream)))
        return grads

    def render_fullframe(self, scene, cams: np.ndarray, out=None, stream=None) -> Tuple[object, Dict]:
        """The full-frame baseline: every view rendered whole, then interlaced."""
        out = self._image(out)
        g = gaussians_struct(scene)
        carr, n = cameras_array(cams)
        st = CStats()
        _check(load().lfd_render_fullframe(self._h, ct.byref(g), carr, n, _dptr(out),
                                           _stream_ptr(stream), ct.byref(st)))
        return out, st.as_dict()

    def render_host(self, scene_host, cams: np.ndarray, out_host, stream=None):
        """scene_host / out_host: contiguous CPU tensors (pinned for speed)."""
        g = gaussians_struct(scene_host, host=True)
        carr, n = cameras_array(cams)
        st = CStats()
        _check(load().lfd_render_host(self._h, ct.byref(g), carr, n, out_host.data_ptr(),
                                      _stream_ptr(stream), ct.byref(st)))
        return out_host, st.as_dict()

    def render_host_async(self, scene_host, cams: np.ndarray, out_host, stream=None):
        """lfd_render_host_async: queue a frame; out_host is filled by the time
        render_host_wait() returns. The host tensors are kept alive until then."""
        g = gaussians_struct(scene_host, host=True)
        carr, n = cameras_array(cams)
        st = CStats()
        self._pending.append((scene_host, out_host, carr))
        _check(load().lfd_render_host_async(self._h, ct.byref(g), carr, n, out_host.data_ptr(),
                                            _stream_ptr(stream), ct.byref(st)))
        return out_host, st.as_dict()

    def render_host_wait(self):
        """lfd_render_host_wait: every queued frame's image is in host memory."""
        try:
            _check(load().lfd_render_host_wait(self._h))
        finally:
            self._pending = []

    def reserve(self, max_gaussians: int, max_pairs: int):
        """lfd_plan_reserve: capacity mode (no read-back; graph-capturable
        frames). max_pairs = 0 leaves capacity mode."""
        _check(load().lfd_plan_reserve(self._h, int(max_gaussians), int(max_pairs)))

    def status(self) -> int:
        """lfd_plan_status: raises LFDError on overflow / wait timeout;
        returns the last frame's pair count."""
        P = ct.c_int64(0)
        _check(load().lfd_plan_status(self._h, ct.byref(P)))
        return int(P.value)

    def status_code(self) -> Tuple[int, int]:
        """(status code, last pair count) of lfd_plan_status, without raising."""
        P = ct.c_int64(0)
        rc = load().lfd_plan_status(self._h, ct.byref(P))
        return rc, int(P.value)

    def stage_totals(self, reset: bool = False) -> Dict[str, float]:
        t = CStageTotals()
        _check(load().lfd_get_stage_totals(self._h, ct.byref(t), 1 if reset else 0))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def lists(self, num_pairs: int, with_keys: bool = False):
        lst = np.zeros(max(num_pairs, 1), np.uint32)
        ranges = np.zeros((self.T, self.K, 2), np.uint32)
        keys = np.zeros(max(num_pairs, 1), np.uint64) if with_keys else None
        _check(load().lfd_plan_copy_lists(self._h, lst.ctypes.data, ranges.ctypes.data,
                                          keys.ctypes.data if with_keys else None,
                                          max(num_pairs, 1)))
        return lst[:num_pairs], ranges, (keys[:num_pairs] if with_keys else None)


def measure_alu_peaks(stream=None) -> Dict[str, float]:
    """lfd_measure_alu_peaks: measured FP32 lane operations/s and exp2/s."""
    f, e = ct.c_double(), ct.c_double()
    _check(load().lfd_measure_alu_peaks(ct.byref(f), ct.byref(e), _stream_ptr(stream)))
    return {"fp32_ops_per_s": f.value, "ex2_per_s": e.value}


def make_arc_cameras(num_views: int, cone_deg: float, radius: float, fov_x_deg: float,
                     width: int, height: int) -> np.ndarray:
    """lfd_make_arc_cameras: the display's view cone as num_views pinhole
    cameras; float32 [num_views, 16] rows (R[9], t[3], fx, fy, cx, cy)."""
    arr = (CCamera * num_views)()
    _check(load().lfd_make_arc_cameras(int(num_views), float(cone_deg), float(radius), float(fov_x_deg),
                                       int(width), int(height), arr))
    return np.ctypeslib.as_array(ct.cast(arr, ct.POINTER(ct.c_float)),
                                 shape=(num_views, 16)).copy()


def kernel_launches() -> int:
    """Kernels launched by liblfd in this process so far."""
    return int(load().lfd_kernel_launches())


def scene_to_device(scene: Dict[str, np.ndarray], device="cuda", attr_dtype=None):
    """Scene arrays to device tensors; means stay FP32, the other attributes
    are cast to attr_dtype (a torch dtype: float32, float16 or bfloat16)."""
    import torch
    out = {}
    for k, v in scene.items():
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(device)
        if k != "means" and attr_dtype is not None:
            t = t.to(attr_dtype).contiguous()
        out[k] = t
    return out


def render_autograd(plan: "Plan", cams: np.ndarray, means, scales, quats, opacities, sh,
                    keep_state: bool = True):
    """Differentiable interlaced render: forward through lfd_render, backward
    through lfd_render_backward (a torch.autograd.Function). keep_state turns
    on the plan's FLAG_KEEP_BLEND_STATE so that the backward starts from each
    subpixel's final transmittance and stop position kept by the forward
    (8 bytes per subpixel); without it (and the flag off) the backward
    re-blends every (tile, cluster) list first. Either way no per-subpixel
    list is stored: the backward walks the tile lists again."""
    import torch

    want = (plan.flags | FLAG_KEEP_BLEND_STATE) if keep_state else (plan.flags & ~FLAG_KEEP_BLEND_STATE)
    if want != plan.flags:
        plan.set_flags(want)

    class _Render(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m, s, q, o, h):
            scene = {"means": m.contiguous(), "scales": s.contiguous(), "quats": q.contiguous(),
                     "opacities": o.contiguous(), "sh": h.contiguous()}
            img, _ = plan.render(scene, cams)
            ctx.scene = scene
            return img

        @staticmethod
        def backward(ctx, grad_img):
            g = plan.backward(ctx.scene, cams, grad_img.contiguous())
            return g["means"], g["scales"], g["quats"], g["opacities"], g["sh"]

    return _Render.apply(means, scales, quats, opacities, sh)


class Batch:
    """Several scenes rendered per frame (lfd_batch_*): plans[s] gives scene
    s's panel; plans may repeat. Always in capacity mode (reserve first)."""

    def __init__(self, plans):
        L = load()
        self.plans = list(plans)  # keeps the plans alive for the batch
        arr = (_P * len(self.plans))(*[p._h for p in self.plans])
        h = _P()
        _check(L.lfd_batch_create(arr, len(self.plans), ct.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().lfd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, max_gaussians, max_pairs: int):
        arr = (ct.c_int64 * len(self.plans))(*[int(m) for m in max_gaussians])
        _check(load().lfd_batch_reserve(self._h, arr, int(max_pairs)))

    def images(self):
        import torch
        return [torch.empty((p.panel.height, p.panel.width, 3), dtype=torch.float32, device="cuda")
                for p in self.plans]

    def render(self, scenes, cams_list, outs=None, stream=None):
        """scenes: list of device scene dicts; cams_list: list of [N_s, 16]
        float32 camera arrays. Returns the list of images (no sync)."""
        n = len(self.plans)
        outs = outs if outs is not None else self.images()
        gs = (CGaussians * n)(*[gaussians_struct(sc) for sc in scenes])
        carrs = [cameras_array(c)[0] for c in cams_list]
        self._keep = carrs  # the host arrays must live through the call
        cptrs = (_P * n)(*[ct.cast(a, _P) for a in carrs])
        optrs = (_P * n)(*[_dptr(o) for o in outs])
        _check(load().lfd_batch_render(self._h, ct.cast(gs, _P), ct.cast(cptrs, _P),
                                       ct.cast(optrs, _P), _stream_ptr(stream)))
        return outs

    def status(self) -> int:
        P = ct.c_int64(0)
        _check(load().lfd_batch_status(self._h, ct.byref(P)))
        return int(P.value)

    def status_code(self) -> Tuple[int, int]:
        P = ct.c_int64(0)
        rc = load().lfd_batch_status(self._h, ct.byref(P))
        return rc, int(P.value)
