"""ctypes binding of liblumipath.so (C ABI in include/lumipath.h).

Argument marshalling only: every step of the light-field sampling path runs in
the library's CUDA kernels. Functions keep the C names (``lf_create_table``,
``lf_render``, ``lf_render_backward``, ``lf_destroy`` ...) and take raw device
pointers (ints) and a CUDA stream handle; a non-OK status raises ``LfError``
with the library's message. ``torch_api`` builds the tensor-level API on top.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

from . import build as _build

LF_OK, LF_ERR_INVALID_ARG, LF_ERR_OUT_OF_MEMORY, LF_ERR_CUDA = 0, 1, 2, 3
LF_ERR_UNSUPPORTED, LF_ERR_TIMEOUT, LF_ERR_DEVICE_CHECK = 4, 5, 6
LF_DTYPE_F32, LF_DTYPE_F16, LF_DTYPE_E4M3 = 0, 1, 2
LF_TABLE_BORROW = 0x1
LF_TABLE_UPPER_HEMISPHERE = 0x2
DTYPES = {"f32": LF_DTYPE_F32, "f16": LF_DTYPE_F16, "e4m3": LF_DTYPE_E4M3}


class LfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lumipath status {status}: {msg}")
        self.status = status


class lf_table_desc(C.Structure):
    _fields_ = [("radius", C.c_double), ("center", C.c_double * 3), ("n_origins", C.c_uint32),
                ("n_directions", C.c_uint32), ("channels", C.c_uint32), ("dtype", C.c_int32),
                ("flags", C.c_uint32), ("k_nearest", C.c_uint32)]


class lf_view(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("forward", C.c_float * 3), ("tan_half_x", C.c_float), ("tan_half_y", C.c_float),
                ("width", C.c_uint32), ("height", C.c_uint32), ("out_offset", C.c_uint64)]


class lf_launch(C.Structure):
    _fields_ = [("tile_w", C.c_uint32), ("tile_h", C.c_uint32), ("warp_w", C.c_uint32),
                ("order", C.c_uint32), ("persistent", C.c_uint32), ("ctas_per_sm", C.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class lf_blob(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("width", C.c_float), ("density", C.c_float),
                ("emit", C.c_float * 3)]


class lf_precompute_desc(C.Structure):
    _fields_ = [("radius", C.c_double), ("center", C.c_double * 3), ("n_origins", C.c_uint32),
                ("n_directions", C.c_uint32), ("channels", C.c_uint32), ("rows", C.c_uint32),
                ("spp", C.c_uint32), ("steps", C.c_uint32), ("jitter", C.c_uint32),
                ("n_blobs", C.c_uint32), ("seed", C.c_uint64), ("bg0", C.c_float * 3),
                ("bg1", C.c_float * 3)]


LF_PRECOMPUTE_MAX_BLOBS = 16

_lib = None
_lock = threading.Lock()


def lib():
    """Load liblumipath.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("LUMIPATH_LIB")      # another build of the library (e.g. debug)
            if not path:
                path = _build.LIB
                if not _build.up_to_date():
                    path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"liblumipath.so is missing at {path}")
            L = C.CDLL(path)
            vp, u32, i32, u64, st = C.c_void_p, C.c_uint32, C.c_int32, C.c_uint64, C.c_int
            sig = {
                "lf_create_table": (st, [C.POINTER(lf_table_desc), vp, vp, vp, C.POINTER(vp)]),
                "lf_render": (st, [vp, C.POINTER(lf_view), u32, vp, vp, vp]),
                "lf_render_f16": (st, [vp, C.POINTER(lf_view), u32, vp, vp, vp]),
                "lf_render_backward": (st, [vp, C.POINTER(lf_view), u32, vp, vp, vp]),
                "lf_render_backward_idx": (st, [vp, C.POINTER(lf_view), u32, vp, vp, vp, vp]),
                "lf_destroy": (None, [vp]),
                "lf_last_error": (C.c_char_p, []),
                "lf_set_launch": (st, [vp, C.POINTER(lf_launch)]),
                "lf_get_launch": (st, [vp, C.POINTER(lf_launch)]),
                "lf_sync_status": (st, [vp, vp]),
                "lf_quantize_table": (st, [vp, u32, u32, u32, i32, vp, vp, vp]),
                "lf_fill_lobe_table": (st, [u32, u32, u32, u32, vp, vp, vp, vp, vp, u64, vp, vp]),
                "lf_device_sm_count": (C.c_int, []),
                "lf_version": (C.c_char_p, []),
                "lf_struct_size": (C.c_size_t, [C.c_int]),
                "lf_render_noalloc": (st, [C.POINTER(lf_table_desc), vp, vp, C.POINTER(lf_view), u32,
                                           C.POINTER(lf_launch), vp, vp, vp]),
                "lf_noalloc_sync_status": (st, [vp]),
                "lf_precompute_table": (st, [C.POINTER(lf_precompute_desc), C.POINTER(lf_blob), vp, vp]),
                "lf_render_volume": (st, [C.POINTER(lf_precompute_desc), C.POINTER(lf_blob),
                                          C.POINTER(lf_view), u32, vp, vp]),
                "lf_post_filter": (st, [C.c_double, C.POINTER(C.c_double), u32, vp, C.POINTER(lf_view), u32,
                                        vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            for k, s in enumerate((lf_table_desc, lf_view, lf_launch, lf_precompute_desc, lf_blob)):
                if L.lf_struct_size(k) != C.sizeof(s):
                    raise RuntimeError(f"ABI mismatch: {s.__name__} is {C.sizeof(s)} bytes here, "
                                       f"{L.lf_struct_size(k)} in the library")
            _lib = L
    return _lib


def _check(status: int):
    if status != LF_OK:
        raise LfError(status, lib().lf_last_error().decode(errors="replace"))


def make_views(views: Sequence) -> "C.Array":
    """lf_view array from objects with eye/right/up/forward/tan_half_x/
    tan_half_y/width/height/out_offset attributes (e.g. lf_inputs.View)."""
    arr = (lf_view * len(views))()
    for k, v in enumerate(views):
        a = arr[k]
        a.eye[:] = list(v.eye)
        a.right[:] = list(v.right)
        a.up[:] = list(v.up)
        a.forward[:] = list(v.forward)
        a.tan_half_x = v.tan_half_x
        a.tan_half_y = v.tan_half_y
        a.width = v.width
        a.height = v.height
        a.out_offset = v.out_offset
    return arr


# ---------------------------------------------------------------------------
# Entry points under their C names
# ---------------------------------------------------------------------------
def lf_create_table(desc: lf_table_desc, radiance_ptr: int, scales_ptr: Optional[int],
                    stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().lf_create_table(C.byref(desc), C.c_void_p(radiance_ptr),
                                 C.c_void_p(scales_ptr or None), C.c_void_p(stream or None), C.byref(h)))
    return int(h.value)


def lf_render(table: int, views, n_views: int, out_ptr: int, idx_ptr: Optional[int], stream: int = 0):
    _check(lib().lf_render(C.c_void_p(table), views, n_views, C.c_void_p(out_ptr),
                           C.c_void_p(idx_ptr or None), C.c_void_p(stream or None)))


def lf_render_f16(table: int, views, n_views: int, out_ptr: int, idx_ptr: Optional[int], stream: int = 0):
    _check(lib().lf_render_f16(C.c_void_p(table), views, n_views, C.c_void_p(out_ptr),
                               C.c_void_p(idx_ptr or None), C.c_void_p(stream or None)))


def lf_render_backward(table: int, views, n_views: int, grad_out_ptr: int, grad_table_ptr: int,
                       stream: int = 0):
    _check(lib().lf_render_backward(C.c_void_p(table), views, n_views, C.c_void_p(grad_out_ptr),
                                    C.c_void_p(grad_table_ptr), C.c_void_p(stream or None)))


def lf_render_backward_idx(table: int, views, n_views: int, grad_out_ptr: int, idx_ptr: int,
                           grad_table_ptr: int, stream: int = 0):
    _check(lib().lf_render_backward_idx(C.c_void_p(table), views, n_views, C.c_void_p(grad_out_ptr),
                                        C.c_void_p(idx_ptr), C.c_void_p(grad_table_ptr),
                                        C.c_void_p(stream or None)))


def lf_destroy(table: Optional[int]):
    if table:
        lib().lf_destroy(C.c_void_p(table))


def lf_last_error() -> str:
    return lib().lf_last_error().decode(errors="replace")


def lf_set_launch(table: int, cfg: lf_launch):
    _check(lib().lf_set_launch(C.c_void_p(table), C.byref(cfg)))


def lf_get_launch(table: int) -> lf_launch:
    cfg = lf_launch()
    _check(lib().lf_get_launch(C.c_void_p(table), C.byref(cfg)))
    return cfg


def lf_sync_status(table: int, stream: int = 0):
    _check(lib().lf_sync_status(C.c_void_p(table), C.c_void_p(stream or None)))


def lf_quantize_table(src_ptr: int, M: int, N: int, Cc: int, dtype: int, codes_ptr: int,
                      scales_ptr: int, stream: int = 0):
    _check(lib().lf_quantize_table(C.c_void_p(src_ptr), M, N, Cc, dtype, C.c_void_p(codes_ptr),
                                   C.c_void_p(scales_ptr), C.c_void_p(stream or None)))


def lf_fill_lobe_table(M: int, N: int, Cc: int, L: int, ap, ad, kp, kd, col, noise_seed: int,
                       out_ptr: int, stream: int = 0):
    import numpy as np
    arrs = [np.ascontiguousarray(a, np.float64) for a in (ap, ad, kp, kd, col)]
    ptrs = [a.ctypes.data_as(C.c_void_p) if a.size else None for a in arrs]
    _check(lib().lf_fill_lobe_table(M, N, Cc, L, *ptrs, C.c_uint64(noise_seed & (2**64 - 1)),
                                    C.c_void_p(out_ptr), C.c_void_p(stream or None)))


def lf_render_noalloc(desc: lf_table_desc, radiance_ptr: int, scales_ptr: Optional[int], views,
                      n_views: int, launch: Optional[lf_launch], out_ptr: int, idx_ptr: Optional[int],
                      stream: int = 0):
    """Render straight from the caller's arrays; the library allocates nothing
    (for callers that cannot call cudaMalloc; see include/lumipath.h)."""
    _check(lib().lf_render_noalloc(C.byref(desc), C.c_void_p(radiance_ptr), C.c_void_p(scales_ptr or None),
                                   views, n_views, C.byref(launch) if launch is not None else None,
                                   C.c_void_p(out_ptr), C.c_void_p(idx_ptr or None),
                                   C.c_void_p(stream or None)))


def lf_noalloc_sync_status(stream: int = 0):
    """Synchronise the stream and raise LfError(LF_ERR_DEVICE_CHECK) if a kernel of
    the last lf_render_noalloc call on this device recorded a failed device check."""
    _check(lib().lf_noalloc_sync_status(C.c_void_p(stream or None)))


def lf_precompute_table(desc: lf_precompute_desc, blobs, out_ptr: int, stream: int = 0):
    """Light-field precompute of a volume scene into a device FP32 table (Section 2)."""
    _check(lib().lf_precompute_table(C.byref(desc), blobs, C.c_void_p(out_ptr), C.c_void_p(stream or None)))


def lf_render_volume(desc: lf_precompute_desc, blobs, views, n_views: int, out_ptr: int, stream: int = 0):
    """Direct render of the precompute's volume along each pixel's ray (the
    ground truth of a light-field render of the precomputed table)."""
    _check(lib().lf_render_volume(C.byref(desc), blobs, views, n_views, C.c_void_p(out_ptr),
                                  C.c_void_p(stream or None)))


LF_POST_WEIGHTS = 3347


def lf_post_filter(radius: float, center, channels: int, weights_host, views, n_views: int, in_ptr: int,
                   out_ptr: int, stream: int = 0):
    """Learned post-filter of a light-field image (three 3x3 convolution layers,
    residual on hit pixels); weights_host: a ctypes array of LF_POST_WEIGHTS floats."""
    c = (C.c_double * 3)(*[float(x) for x in center])
    _check(lib().lf_post_filter(float(radius), c, channels, weights_host, views, n_views,
                                C.c_void_p(in_ptr), C.c_void_p(out_ptr), C.c_void_p(stream or None)))


def lf_device_sm_count() -> int:
    return int(lib().lf_device_sm_count())


def lf_version() -> str:
    return lib().lf_version().decode()
