"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/lumipath.h declares, agrees with the binding on structure
layouts, and rejects bad arguments with a status (never an abort) before any
device work."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1903_03837_gb300 import build as B
from paper_1903_03837_gb300 import lumipath as lp

HEADER = os.path.join(B.INCLUDE, "lumipath.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = lp.lib()
    names = declared_functions()
    assert {"lf_create_table", "lf_render", "lf_render_backward", "lf_destroy"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lf_[a-z0-9_]+)$", out, flags=re.M))
    for n in names:
        assert n in exported, n
        assert getattr(lib, n) is not None


def test_struct_layouts_match():
    L = lp.lib()
    assert L.lf_struct_size(0) == C.sizeof(lp.lf_table_desc) == 56
    assert L.lf_struct_size(1) == C.sizeof(lp.lf_view) == 72
    assert L.lf_struct_size(2) == C.sizeof(lp.lf_launch) == 24
    assert L.lf_struct_size(3) == C.sizeof(lp.lf_precompute_desc) == 96
    assert L.lf_struct_size(4) == C.sizeof(lp.lf_blob) == 32
    assert L.lf_struct_size(7) == 0


def test_built_for_sm_103a_only():
    flags = " ".join(B.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert flags.count("-gencode") == 1


def _desc(**kw):
    d = lp.lf_table_desc()
    d.radius = kw.get("radius", 1.0)
    d.center[:] = kw.get("center", [0.0, 0.0, 0.0])
    d.n_origins = kw.get("M", 64)
    d.n_directions = kw.get("N", 32)
    d.channels = kw.get("C", 4)
    d.dtype = kw.get("dtype", 0)
    d.flags = kw.get("flags", 0)
    d.k_nearest = kw.get("k", 0)
    return d


@pytest.mark.parametrize("kw,status", [
    (dict(radius=0.0), lp.LF_ERR_INVALID_ARG),
    (dict(radius=-1.0), lp.LF_ERR_INVALID_ARG),
    (dict(radius=float("nan")), lp.LF_ERR_INVALID_ARG),
    (dict(center=[0.0, float("inf"), 0.0]), lp.LF_ERR_INVALID_ARG),
    (dict(M=0), lp.LF_ERR_INVALID_ARG),
    (dict(N=0), lp.LF_ERR_INVALID_ARG),
    (dict(M=(1 << 24) + 1), lp.LF_ERR_INVALID_ARG),
    (dict(C=2), lp.LF_ERR_INVALID_ARG),
    (dict(C=5), lp.LF_ERR_INVALID_ARG),
    (dict(dtype=7), lp.LF_ERR_INVALID_ARG),
    (dict(dtype=1), lp.LF_ERR_INVALID_ARG),          # F16 without scales
    (dict(flags=0x80), lp.LF_ERR_INVALID_ARG),
    (dict(k=7), lp.LF_ERR_UNSUPPORTED),
    (dict(k=16), lp.LF_ERR_UNSUPPORTED),
])
def test_create_table_rejects_bad_descriptions(kw, status):
    h = C.c_void_p(123)
    d = _desc(**kw)
    s = lp.lib().lf_create_table(C.byref(d), C.c_void_p(0x1000), None, None, C.byref(h))
    assert s == status
    assert h.value is None
    assert lp.lf_last_error() != ""


def test_null_arguments_are_errors_not_crashes():
    L = lp.lib()
    h = C.c_void_p()
    assert L.lf_create_table(None, C.c_void_p(0x1000), None, None, C.byref(h)) == lp.LF_ERR_INVALID_ARG
    d = _desc()
    assert L.lf_create_table(C.byref(d), None, None, None, C.byref(h)) == lp.LF_ERR_INVALID_ARG
    assert L.lf_create_table(C.byref(d), C.c_void_p(0x1000), None, None, None) == lp.LF_ERR_INVALID_ARG
    views = lp.make_views([])
    assert L.lf_render(None, views, 0, C.c_void_p(0x1000), None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_render_backward(None, views, 0, None, None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_set_launch(None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_sync_status(None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_quantize_table(None, 4, 4, 4, 1, None, None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_quantize_table(C.c_void_p(16), 4, 4, 4, 0, C.c_void_p(16), C.c_void_p(16), None) \
        == lp.LF_ERR_INVALID_ARG
    assert L.lf_fill_lobe_table(4, 4, 4, 65, None, None, None, None, None, 0, C.c_void_p(16), None) \
        == lp.LF_ERR_INVALID_ARG
    L.lf_destroy(None)


def test_error_message_is_thread_local():
    import threading
    L = lp.lib()
    h = C.c_void_p()
    d = _desc(C=9)
    L.lf_create_table(C.byref(d), C.c_void_p(0x1000), None, None, C.byref(h))
    mine = lp.lf_last_error()
    seen = []
    t = threading.Thread(target=lambda: seen.append(lp.lf_last_error()))
    t.start()
    t.join()
    assert "channels" in mine and seen == [""]


def _pdesc(**kw):
    d = lp.lf_precompute_desc()
    d.radius = kw.get("radius", 1.0)
    d.center[:] = kw.get("center", [0.0, 0.0, 0.0])
    d.n_origins = kw.get("M", 64)
    d.n_directions = kw.get("N", 32)
    d.channels = kw.get("C", 4)
    d.rows = kw.get("rows", d.n_origins)
    d.spp = kw.get("spp", 4)
    d.steps = kw.get("steps", 16)
    d.jitter = kw.get("jitter", 1)
    d.n_blobs = kw.get("nb", 1)
    d.seed = 1
    d.bg0[:] = kw.get("bg0", [0.0, 0.0, 0.0])
    d.bg1[:] = [0.0, 0.0, 0.0]
    return d


def _blobs(width=0.2, density=3.0, n=1):
    b = (lp.lf_blob * max(n, 1))()
    for k in range(n):
        b[k].center[:] = [0.0, 0.0, 0.0]
        b[k].width = width
        b[k].density = density
        b[k].emit[:] = [1.0, 0.5, 0.25]
    return b


@pytest.mark.parametrize("kw,blob", [
    (dict(M=0), {}), (dict(N=1 << 25), {}), (dict(radius=0.0), {}), (dict(radius=float("nan")), {}),
    (dict(C=2), {}), (dict(rows=0), {}), (dict(rows=65), {}), (dict(spp=0), {}), (dict(spp=2000), {}),
    (dict(steps=0), {}), (dict(steps=5000), {}), (dict(jitter=2), {}), (dict(nb=17), {}),
    (dict(bg0=[float("inf"), 0.0, 0.0]), {}), ({}, dict(width=0.0)), ({}, dict(width=-1.0)),
    ({}, dict(density=-0.5)), ({}, dict(density=float("nan"))),
])
def test_precompute_rejects_bad_arguments(kw, blob):
    # validation happens before any CUDA call; the fake output pointer is never touched
    L = lp.lib()
    d = _pdesc(**kw)
    st = L.lf_precompute_table(C.byref(d), _blobs(n=max(1, d.n_blobs), **blob), C.c_void_p(4096), None)
    assert st == lp.LF_ERR_INVALID_ARG, (kw, blob, lp.lf_last_error())
    assert lp.lf_last_error()


def test_precompute_null_and_misaligned_arguments():
    L = lp.lib()
    d = _pdesc()
    assert L.lf_precompute_table(None, _blobs(), C.c_void_p(4096), None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_precompute_table(C.byref(d), _blobs(), None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_precompute_table(C.byref(d), None, C.c_void_p(4096), None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_precompute_table(C.byref(d), _blobs(), C.c_void_p(4100), None) == lp.LF_ERR_INVALID_ARG
    assert "aligned" in lp.lf_last_error()


@pytest.mark.parametrize("dtype,Cc,ptr", [(0, 4, 0x1008), (0, 3, 0x1004), (1, 4, 0x1004), (2, 4, 0x1002)])
def test_borrowed_table_must_be_aligned_for_its_vector_loads(dtype, Cc, ptr):
    # float4 (F32 RGBA), float2 + float (F32 RGB), uint2 (F16), uint32 (E4M3) texel loads:
    # a misaligned pointer is an argument error before any device work
    d = _desc(C=Cc, dtype=dtype, flags=lp.LF_TABLE_BORROW)
    handle = C.c_void_p()
    s = lp.lib().lf_create_table(C.byref(d), C.c_void_p(ptr), C.c_void_p(0x2000), None, C.byref(handle))
    assert s == lp.LF_ERR_INVALID_ARG, lp.lf_last_error()
    assert "aligned" in lp.lf_last_error()
    assert handle.value is None


def _one_view():
    import lf_inputs
    return lp.make_views([lf_inputs.look_at((2.5, 0.3, 0.2), (0, 0, 0), 8, 8)])


@pytest.mark.parametrize("kw,blob", [
    (dict(radius=0.0), {}), (dict(radius=float("nan")), {}), (dict(C=5), {}), (dict(steps=0), {}),
    (dict(steps=5000), {}), (dict(nb=17), {}), (dict(bg0=[float("nan"), 0.0, 0.0]), {}),
    ({}, dict(width=0.0)), ({}, dict(density=-1.0)),
])
def test_render_volume_rejects_bad_volumes(kw, blob):
    # the direct render shares the precompute's volume checks; all before any CUDA call
    L = lp.lib()
    d = _pdesc(**kw)
    st = L.lf_render_volume(C.byref(d), _blobs(n=max(1, d.n_blobs), **blob), _one_view(), 1,
                            C.c_void_p(4096), None)
    assert st == lp.LF_ERR_INVALID_ARG, (kw, blob, lp.lf_last_error())


def test_render_volume_checks_views_and_output_not_the_sets():
    L = lp.lib()
    # the SF-set fields are not used: M = 0, rows = 0, spp = 0 and jitter = 2 pass the
    # volume checks, and the call stops at the (empty) view list instead
    d = _pdesc(M=0, rows=0, spp=0, jitter=2)
    assert L.lf_render_volume(C.byref(d), _blobs(), _one_view(), 0, C.c_void_p(4096), None) == \
        lp.LF_ERR_INVALID_ARG
    assert "n_views" in lp.lf_last_error()
    d = _pdesc()
    assert L.lf_render_volume(None, _blobs(), _one_view(), 1, C.c_void_p(4096), None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_render_volume(C.byref(d), _blobs(), None, 1, C.c_void_p(4096), None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_render_volume(C.byref(d), _blobs(), _one_view(), 1, None, None) == lp.LF_ERR_INVALID_ARG
    assert L.lf_render_volume(C.byref(d), _blobs(), _one_view(), 1, C.c_void_p(4100), None) == \
        lp.LF_ERR_INVALID_ARG
    assert "aligned" in lp.lf_last_error()


def test_post_filter_argument_errors_before_any_device_work():
    L = lp.lib()
    c3 = (C.c_double * 3)(0.0, 0.0, 0.0)
    v = _one_view()                    # 8 x 8 pixels
    W = (C.c_float * lp.LF_POST_WEIGHTS)()
    IN, OUT = C.c_void_p(0x20000), C.c_void_p(0x30000)
    cases = [
        (1.0, None, 4, W, v, 1, IN, OUT), (1.0, c3, 4, None, v, 1, IN, OUT), (1.0, c3, 4, W, v, 1, None, OUT),
        (1.0, c3, 4, W, v, 1, IN, None), (0.0, c3, 4, W, v, 1, IN, OUT), (float("inf"), c3, 4, W, v, 1, IN, OUT),
        (1.0, c3, 5, W, v, 1, IN, OUT), (1.0, c3, 4, W, v, 0, IN, OUT), (1.0, c3, 4, W, None, 1, IN, OUT),
        (1.0, c3, 4, W, v, 1, C.c_void_p(0x20002), OUT),
        (1.0, c3, 4, W, v, 1, IN, C.c_void_p(0x20000 + 64 * 16 - 4)),      # out overlaps in's last pixel
    ]
    for args in cases:
        assert L.lf_post_filter(*args, None) == lp.LF_ERR_INVALID_ARG, (args, lp.lf_last_error())
    assert "overlap" in lp.lf_last_error()
    W[7] = float("nan")
    assert L.lf_post_filter(1.0, c3, 4, W, v, 1, IN, OUT, None) == lp.LF_ERR_INVALID_ARG
    assert "finite" in lp.lf_last_error()
