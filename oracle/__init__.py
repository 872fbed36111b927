"""CPU oracle of the LumiPath light-field sampling path (arXiv 1903.03837).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library (``paper_1903_03837_gb300``) and does not import it; the
two meet only in the seeded inputs of ``lf_inputs``.

The arithmetic lives in ``lf_oracle.c`` (plain C, FP64 for every quantity
that decides a neighbour; see that file's header for the paper passage each
function follows). This wrapper compiles it with gcc on first use and
marshals numpy arrays through ctypes. Functions:

* ``sf_phase``, ``sf_point``, ``sf_points``  -- SF point set, Section 2 equation
* ``camera_ray``, ``trace_pixel``            -- pinhole ray and sphere hits, Section 2
* ``knn``                                    -- brute-force K nearest SF points
* ``kernel_sigma``, ``tent_weights``         -- distance filter kernel, Section 2
* ``render_pixels``, ``render_views``        -- 25-tap blend (K=5), Section 2
* ``render_backward``                        -- adjoint of the blend w.r.t. the table
* ``f16_*``, ``e4m3_*``, ``quantize_rows``   -- per-row FP16 / E4M3 table storage
* ``lobe_table``                             -- the synthetic lobe radiance field
* ``volume_table``, ``volume_ray``, ``volume_origin`` -- light-field precompute (Section 2):
  every ray r_k through an emission-absorption volume of Gaussian blobs, origins
  jittered on the disk of area A_S/M
* ``volume_pixels``                          -- direct render of that volume along each
  pixel's ray (the ground truth of a light-field render of the precomputed table)
* ``post_filter``, ``post_features``, ``conv3x3`` -- the learned post-filter's forward
  (Section 2, post-processing) in FP64
* ``psnr``                                   -- image error against an FP64 render

Parity unpinned: none. Each function is pinned against facts that do not come
from the oracle (closed forms, brute force, library routines, invariants) in
``tests/test_oracle_pins.py`` (sampling path), ``tests/test_oracle_volume.py``
(precompute and direct render) and ``tests/test_oracle_post.py`` (post-filter).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblf_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fno-math-errno"]


def build(force: bool = False) -> str:
    """Compile lf_oracle.c into _build/liblf_oracle.so (gcc, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Lobes(C.Structure):
    _fields_ = [("L", C.c_uint32), ("C", C.c_uint32), ("seed", C.c_uint64),
                ("ap", C.c_void_p), ("ad", C.c_void_p), ("kp", C.c_void_p),
                ("kd", C.c_void_p), ("col", C.c_void_p)]


class _Scene(C.Structure):
    _fields_ = [("R", C.c_double), ("O", C.c_double * 3), ("M", C.c_uint32),
                ("N", C.c_uint32), ("C", C.c_uint32), ("K", C.c_int),
                ("Po", C.c_void_p), ("Pd", C.c_void_p), ("dtype", C.c_int),
                ("table", C.c_void_p), ("scales", C.c_void_p), ("lobes", C.c_void_p),
                ("rowmap", C.c_void_p), ("upper", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, u32, u64, i64, dbl = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64, C.c_double
            sig = {
                "lfo_sf_phase": (dbl, [u64]),
                "lfo_sf_point": (None, [u32, u32, vp]),
                "lfo_sf_points": (None, [u32, vp]),
                "lfo_camera_ray": (None, [vp, u32, u32, u32, u32, vp]),
                "lfo_intersect": (C.c_int, [C.c_float, vp, vp, vp, vp, vp]),
                "lfo_normalize_hit": (None, [vp, vp, vp]),
                "lfo_knn": (C.c_int, [vp, u32, vp, C.c_int, vp, vp]),
                "lfo_kernel_sigma": (dbl, [u32]),
                "lfo_tent_weights": (None, [vp, C.c_int, u32, vp]),
                "lfo_tent_weights_kept": (None, [vp, vp, C.c_int, u32, C.c_int32, vp]),
                "lfo_f16_decode": (dbl, [C.c_uint16]),
                "lfo_f16_encode": (C.c_uint16, [C.c_float]),
                "lfo_e4m3_decode": (dbl, [C.c_uint8]),
                "lfo_e4m3_encode": (C.c_uint8, [C.c_float]),
                "lfo_quantize_rows": (None, [vp, u32, u32, u32, C.c_int, vp, vp]),
                "lfo_splitmix64": (u64, [u64, u64]),
                "lfo_lobe_texel": (None, [vp, vp, vp, u32, u32, vp]),
                "lfo_lobe_table_rows": (None, [vp, vp, vp, u32, u32, u32, vp]),
                "lfo_render_pixels": (i64, [vp, vp, vp, vp, i64, vp, vp]),
                "lfo_render_backward_pixels": (None, [vp, vp, vp, vp, i64, vp, vp]),
                "lfo_trace_pixel": (C.c_int, [dbl, vp, vp, u32, u32, u32, u32, vp, vp, vp, vp, vp]),
                "lfo_lobe_continuous": (None, [vp, vp, vp, vp]),
                "lfo_lobe_reference_pixels": (i64, [vp, dbl, vp, vp, vp, vp, i64, vp, vp]),
                "lfo_volume_origin": (None, [vp, u32, u32, vp, u32, u32, u32, vp]),
                "lfo_volume_tend": (dbl, [vp, vp, vp]),
                "lfo_volume_ray": (None, [vp, vp, vp, vp, vp]),
                "lfo_volume_texel": (None, [vp, vp, vp, u32, u32, u32, u32, vp]),
                "lfo_volume_table_rows": (None, [vp, vp, vp, u32, u32, u32, u32, vp]),
                "lfo_volume_pixels": (i64, [vp, vp, vp, vp, i64, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _threads(n: Optional[int]) -> int:
    return max(1, int(n if n else (os.cpu_count() or 1)))


# --------------------------------------------------------------------------
# SF points, camera, intersection, k-NN, weights
# --------------------------------------------------------------------------
def sf_phase(i: int) -> float:
    return lib().lfo_sf_phase(int(i))


def sf_point(n: int, i: int) -> np.ndarray:
    p = np.zeros(3)
    lib().lfo_sf_point(n, i, _p(p))
    return p


_points_cache = {}


def sf_points(n: int) -> np.ndarray:
    """[n,3] FP64 SF points (cached; read-only)."""
    P = _points_cache.get(n)
    if P is None:
        P = np.zeros((n, 3))
        lib().lfo_sf_points(n, _p(P))
        P.setflags(write=False)
        _points_cache[n] = P
    return P


def camera_ray(view, x: int, y: int) -> np.ndarray:
    d = np.zeros(3, np.float32)
    lib().lfo_camera_ray(_p(view.floats14()), view.width, view.height, x, y, _p(d))
    return d


def intersect(R: float, O, e, d):
    O32 = np.asarray(O, np.float32)
    e = np.asarray(e, np.float32)
    d = np.asarray(d, np.float32)
    ho = np.zeros(3, np.float32)
    hd = np.zeros(3, np.float32)
    hit = lib().lfo_intersect(float(np.float32(R)), _p(O32), _p(e), _p(d), _p(ho), _p(hd))
    return bool(hit), ho, hd


def trace_pixel(R: float, O, view, x: int, y: int):
    """(hit, dir, h_o, h_d, q_o, q_d) of one pixel (FP32 ray/hits, FP64 unit hits)."""
    O64 = np.asarray(O, np.float64)
    d = np.zeros(3, np.float32)
    ho = np.zeros(3, np.float32)
    hd = np.zeros(3, np.float32)
    qo = np.zeros(3)
    qd = np.zeros(3)
    hit = lib().lfo_trace_pixel(R, _p(O64), _p(view.floats14()), view.width, view.height,
                                x, y, _p(d), _p(ho), _p(hd), _p(qo), _p(qd))
    return bool(hit), d, ho, hd, qo, qd


def normalize_hit(h, O) -> np.ndarray:
    h = np.asarray(h, np.float32)
    O = np.asarray(O, np.float64)
    q = np.zeros(3)
    lib().lfo_normalize_hit(_p(h), _p(O), _p(q))
    return q


def knn(P: np.ndarray, q, K: int = 5):
    """Brute-force K nearest rows of P to q: (indices, squared distances)."""
    P = np.ascontiguousarray(P, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    idx = np.zeros(16, np.int32)
    d2 = np.zeros(16)
    cnt = lib().lfo_knn(_p(P), P.shape[0], _p(q), K, _p(idx), _p(d2))
    return idx[:cnt].copy(), d2[:cnt].copy()


def kernel_sigma(n: int) -> float:
    return lib().lfo_kernel_sigma(n)


def tent_weights_kept(d2, idx, n: int, rows: int) -> np.ndarray:
    d2 = np.ascontiguousarray(d2, np.float64)
    idx = np.ascontiguousarray(idx, np.int32)
    w = np.zeros(len(d2))
    lib().lfo_tent_weights_kept(_p(d2), _p(idx), len(d2), n, rows, _p(w))
    return w


def tent_weights(d2, n: int) -> np.ndarray:
    d2 = np.ascontiguousarray(d2, np.float64)
    w = np.zeros(len(d2))
    lib().lfo_tent_weights(_p(d2), len(d2), n, _p(w))
    return w


# --------------------------------------------------------------------------
# Quantisers
# --------------------------------------------------------------------------
def f16_decode(codes) -> np.ndarray:
    f = lib().lfo_f16_decode
    return np.array([f(int(c)) for c in np.asarray(codes, np.uint16).ravel()])


def f16_encode(x) -> np.ndarray:
    f = lib().lfo_f16_encode
    return np.array([f(float(v)) for v in np.asarray(x, np.float32).ravel()], np.uint16)


def e4m3_decode(codes) -> np.ndarray:
    f = lib().lfo_e4m3_decode
    return np.array([f(int(c)) for c in np.asarray(codes, np.uint8).ravel()])


def e4m3_encode(x) -> np.ndarray:
    f = lib().lfo_e4m3_encode
    return np.array([f(float(v)) for v in np.asarray(x, np.float32).ravel()], np.uint8)


def quantize_rows(T: np.ndarray, dtype: str):
    """Per-row quantisation of an FP32 [M,N,C] table -> (codes, scales[M])."""
    T = np.ascontiguousarray(T, np.float32)
    M, N, Cc = T.shape
    code_t = {"f16": np.uint16, "e4m3": np.uint8}[dtype]
    codes = np.zeros(T.shape, code_t)
    scales = np.zeros(M, np.float32)
    lib().lfo_quantize_rows(_p(T), M, N, Cc, 1 if dtype == "f16" else 2, _p(codes), _p(scales))
    return codes, scales


def splitmix64(seed: int, ctr: int) -> int:
    return int(lib().lfo_splitmix64(seed & (2**64 - 1), ctr & (2**64 - 1)))


# --------------------------------------------------------------------------
# Lobe field
# --------------------------------------------------------------------------
class _LobesHold:
    def __init__(self, lobes):
        self.ap = np.ascontiguousarray(lobes.ap, np.float64)
        self.ad = np.ascontiguousarray(lobes.ad, np.float64)
        self.kp = np.ascontiguousarray(lobes.kp, np.float64)
        self.kd = np.ascontiguousarray(lobes.kd, np.float64)
        self.col = np.ascontiguousarray(lobes.col, np.float64)
        self.s = _Lobes(lobes.L, lobes.C, lobes.noise_seed, _p(self.ap).value, _p(self.ad).value,
                        _p(self.kp).value, _p(self.kd).value, _p(self.col).value)


def lobe_texel(lobes, M: int, N: int, i: int, j: int) -> np.ndarray:
    h = _LobesHold(lobes)
    out = np.zeros(16)
    lib().lfo_lobe_texel(C.byref(h.s), _p(sf_points(M)), _p(sf_points(N)), i, j, _p(out))
    return out[:lobes.C].copy()


def lobe_continuous(lobes, q, d) -> np.ndarray:
    """The lobe field at origin q (unit) and direction d (unit), without noise."""
    h = _LobesHold(lobes)
    out = np.zeros(16)
    lib().lfo_lobe_continuous(C.byref(h.s), _p(np.ascontiguousarray(q, np.float64)),
                              _p(np.ascontiguousarray(d, np.float64)), _p(out))
    return out[:lobes.C].copy()


def lobe_reference_pixels(lobes, views, pix: np.ndarray, R: float = 1.0, O=(0.0, 0.0, 0.0),
                          threads: Optional[int] = None):
    """Continuous lobe field along each pixel's ray (at the normalised front hit,
    in the chord direction to the back hit): (out [np,C] FP64, hit [np] bool)."""
    h = _LobesHold(lobes)
    vf, wh = _views_arrays(views)
    pix = np.ascontiguousarray(pix, np.uint32)
    out = np.zeros((len(pix), lobes.C))
    hit = np.zeros(len(pix), np.uint8)
    Od = (C.c_double * 3)(*[float(o) for o in O])
    chunks = np.array_split(np.arange(len(pix)), _threads(threads) * 4)

    def work(ch):
        if len(ch):
            a = int(ch[0])
            lib().lfo_lobe_reference_pixels(C.byref(h.s), float(R), Od, _p(vf), _p(wh), _p(pix[a:]),
                                            len(ch), _p(out[a:]), _p(hit[a:]))
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(work, chunks))
    return out, hit.astype(bool)


def lobe_table(lobes, M: int, N: int, rows: Optional[Sequence[int]] = None,
               threads: Optional[int] = None) -> np.ndarray:
    """FP32 table [M,N,C] (or [len(rows),N,C]) of the lobe field, FP64 then rounded."""
    h = _LobesHold(lobes)
    Po, Pd = sf_points(M), sf_points(N)
    L = lib()
    if rows is None:
        out = np.zeros((M, N, lobes.C), np.float32)
        nt = _threads(threads)
        chunks = np.array_split(np.arange(M), nt * 4)

        def work(ch):
            if len(ch):
                L.lfo_lobe_table_rows(C.byref(h.s), _p(Po), _p(Pd), N, int(ch[0]), int(ch[-1]) + 1,
                                      _p(out[ch[0]:]))
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, chunks))
        return out
    rows = [int(r) for r in rows]
    out = np.zeros((len(rows), N, lobes.C), np.float32)

    def one(k):
        L.lfo_lobe_table_rows(C.byref(h.s), _p(Po), _p(Pd), N, rows[k], rows[k] + 1, _p(out[k:]))
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(rows))))
    return out


# --------------------------------------------------------------------------
# Light-field precompute (Section 2): volume scene
# --------------------------------------------------------------------------
class _Volume(C.Structure):
    _fields_ = [("B", C.c_uint32), ("C", C.c_uint32), ("spp", C.c_uint32), ("steps", C.c_uint32),
                ("jitter", C.c_uint32), ("pad_", C.c_uint32), ("seed", C.c_uint64),
                ("R", C.c_double), ("O", C.c_double * 3), ("mu", C.c_void_p), ("width", C.c_void_p),
                ("dens", C.c_void_p), ("emit", C.c_void_p), ("bg0", C.c_double * 3),
                ("bg1", C.c_double * 3)]


class _VolumeHold:
    """ctypes view of a volume scene (any object with mu [B,3], width [B],
    dens [B], emit [B,3], bg0 [3], bg1 [3], spp, steps, jitter, seed, R, O)."""

    def __init__(self, vol, C_: int):
        self.mu = np.ascontiguousarray(np.asarray(vol.mu, np.float64).reshape(-1, 3))
        self.width = np.ascontiguousarray(vol.width, np.float64)
        self.dens = np.ascontiguousarray(vol.dens, np.float64)
        self.emit = np.ascontiguousarray(np.asarray(vol.emit, np.float64).reshape(-1, 3))
        B = len(self.width)
        self.s = _Volume(B, C_, int(vol.spp), int(vol.steps), int(vol.jitter), 0,
                         int(vol.seed) & (2**64 - 1), float(vol.R), (C.c_double * 3)(*vol.O),
                         _p(self.mu).value if B else None, _p(self.width).value if B else None,
                         _p(self.dens).value if B else None, _p(self.emit).value if B else None,
                         (C.c_double * 3)(*vol.bg0), (C.c_double * 3)(*vol.bg1))


def volume_origin(vol, M: int, N: int, i: int, j: int, s: int) -> np.ndarray:
    """Origin of sample s of texel (i, j) (on the tangent disk of area 4 pi R^2 / M)."""
    h = _VolumeHold(vol, 3)
    o = np.zeros(3)
    lib().lfo_volume_origin(C.byref(h.s), M, N, _p(np.ascontiguousarray(sf_point(M, i))), i, j, s, _p(o))
    return o


def volume_ray(vol, o, d):
    """(rgb [3], final transmittance, t_end) of one ray through the volume."""
    h = _VolumeHold(vol, 3)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    rgb, T = np.zeros(3), C.c_double()
    lib().lfo_volume_ray(C.byref(h.s), _p(o), _p(d), _p(rgb), C.byref(T))
    return rgb, T.value, float(lib().lfo_volume_tend(C.byref(h.s), _p(o), _p(d)))


def volume_table(vol, M: int, N: int, C_: int = 4, rows: Optional[Sequence[int]] = None,
                 texels: Optional[np.ndarray] = None, threads: Optional[int] = None) -> np.ndarray:
    """FP32 precomputed table [M,N,C] (or [len(rows),N,C]); with `texels`
    ([K,2] array of (i, j)), FP64 values of those texels [K,C] instead."""
    h = _VolumeHold(vol, C_)
    Po, Pd = sf_points(M), sf_points(N)
    L = lib()
    if texels is not None:
        texels = np.asarray(texels, np.int64).reshape(-1, 2)
        out = np.zeros((len(texels), 4))

        def one_t(k):
            L.lfo_volume_texel(C.byref(h.s), _p(Po), _p(Pd), M, N, int(texels[k, 0]), int(texels[k, 1]),
                               _p(out[k:]))
        with ThreadPoolExecutor(_threads(threads)) as ex:
            list(ex.map(one_t, range(len(texels))))
        return out[:, :C_].copy()
    rows = list(range(M)) if rows is None else [int(r) for r in rows]
    out = np.zeros((len(rows), N, C_), np.float32)

    def one(k):
        L.lfo_volume_table_rows(C.byref(h.s), _p(Po), _p(Pd), M, N, rows[k], rows[k] + 1, _p(out[k:]))
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(one, range(len(rows))))
    return out


def volume_pixels(vol, views, pix: np.ndarray, C_: int = 4, threads: Optional[int] = None):
    """Direct render of the volume at pixels pix [n,3] = (view, x, y): each
    pixel's ray from its front hit on S to the far intersection, one sample,
    no jitter. (out [n,C] FP64 -- RGB, plus opacity 1 - T for C = 4 --, hits);
    misses are 0."""
    h = _VolumeHold(vol, C_)
    pix = np.ascontiguousarray(pix, np.uint32)
    n = pix.shape[0]
    vf, wh = _views_arrays(views)
    out = np.zeros((n, C_))
    L = lib()
    nt = min(_threads(threads), max(1, n // 64))
    bounds = np.linspace(0, n, nt * 4 + 1).astype(np.int64)

    def work(k):
        a, b = int(bounds[k]), int(bounds[k + 1])
        if b <= a:
            return 0
        return L.lfo_volume_pixels(C.byref(h.s), _p(vf), _p(wh), _p(pix[a:]), b - a, _p(out[a:]))
    with ThreadPoolExecutor(nt) as ex:
        hits = sum(ex.map(work, range(len(bounds) - 1)))
    return out, int(hits)


# --------------------------------------------------------------------------
# Learned post-filter (Section 2, post-processing): FP64 forward of the
# three-layer convolutional filter, from the definitions of a 3x3
# cross-correlation with zero padding, ReLU and the residual on hit pixels
# --------------------------------------------------------------------------
POST_SHAPES = [(16, 4, 3, 3), (16,), (16, 16, 3, 3), (16,), (3, 16, 3, 3), (3,)]


def post_unpack(w):
    """(W1, b1, W2, b2, W3, b3) of the flat weight vector (FP64 copies)."""
    w = np.asarray(w, np.float64)
    out, k = [], 0
    for s in POST_SHAPES:
        n = int(np.prod(s))
        out.append(w[k:k + n].reshape(s))
        k += n
    assert k == w.size
    return out


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[o, y, x] = b[o] + sum_{i, dy, dx} W[o, i, dy, dx] in[i, y + dy - 1, x + dx - 1],
    with in = 0 outside the image."""
    I, H, Wd = x.shape
    pad = np.zeros((I, H + 2, Wd + 2))
    pad[:, 1:H + 1, 1:Wd + 1] = x
    out = np.empty((W.shape[0], H, Wd))
    for o in range(W.shape[0]):
        acc = np.full((H, Wd), float(b[o]))
        for i in range(I):
            for dy in range(3):
                for dx in range(3):
                    acc += W[o, i, dy, dx] * pad[i, dy:dy + H, dx:dx + Wd]
        out[o] = acc
    return out


def post_filter(weights, feats: np.ndarray) -> np.ndarray:
    """The filter on one view's features [4, H, W] (R, G, B, hit): [3, H, W] =
    (RGB + conv3(relu(conv2(relu(conv1(feats)))))) on hit pixels, 0 elsewhere."""
    W1, b1, W2, b2, W3, b3 = post_unpack(weights)
    x = np.asarray(feats, np.float64)
    h = np.maximum(conv3x3(x, W1, b1), 0.0)
    h = np.maximum(conv3x3(h, W2, b2), 0.0)
    r = conv3x3(h, W3, b3)
    return (x[:3] + r) * (x[3:4] != 0)


def post_features(view, image: np.ndarray, R: float = 1.0, O=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Features [4, H, W] of one view: the RGB of its [H*W, C] image and the hit
    mask of each pixel's ray (the FP32 ray/sphere test)."""
    H, Wd = view.height, view.width
    f = np.zeros((4, H, Wd))
    img = np.asarray(image, np.float64).reshape(H, Wd, -1)
    f[:3] = img[:, :, :3].transpose(2, 0, 1)
    for y in range(H):
        for x in range(Wd):
            f[3, y, x] = 1.0 if trace_pixel(R, O, view, x, y)[0] else 0.0
    return f


# --------------------------------------------------------------------------
# Rendering
# --------------------------------------------------------------------------
class Scene:
    """Sphere S (R, O), SF set sizes M, N and the table the blend reads.

    table kinds: ``f32`` (FP32 [M,N,C]), ``f16`` / ``e4m3`` (codes [M,N,C] and
    FP32 per-row scales), ``lobe`` (the lobe field evaluated in FP64 on demand).
    With ``rows`` (a list of origin rows), ``table``/``scales`` hold only those
    rows, in that order; reading any other row yields NaN. With ``upper``, only
    the upper-hemisphere origin rows i < M/2 exist (the table has M/2 rows):
    other origin neighbours are dropped and a pixel with none left is masked.
    """

    def __init__(self, M: int, N: int, Cc: int, kind: str = "f32", table=None, scales=None,
                 lobes=None, R: float = 1.0, O=(0.0, 0.0, 0.0), K: int = 5, rows=None,
                 upper: bool = False):
        self.M, self.N, self.C, self.K, self.kind = M, N, Cc, K, kind
        self.R, self.O = float(R), tuple(float(o) for o in O)
        self.Po, self.Pd = sf_points(M), sf_points(N)
        dt = {"f32": 0, "f16": 1, "e4m3": 2, "lobe": 3}[kind]
        tptr = sptr = lptr = rptr = None
        nrows = M // 2 if upper else M
        if rows is not None:
            rows = np.asarray(rows, np.int64)
            nrows = len(rows)
            self.rowmap = np.full(M, -1, np.int32)
            self.rowmap[rows] = np.arange(nrows, dtype=np.int32)
            rptr = _p(self.rowmap).value
        if kind == "f32":
            self.table = np.ascontiguousarray(table, np.float32).reshape(nrows, N, Cc)
            tptr = _p(self.table).value
        elif kind in ("f16", "e4m3"):
            self.table = np.ascontiguousarray(table, np.uint16 if kind == "f16" else np.uint8)
            self.table = self.table.reshape(nrows, N, Cc)
            self.scales = np.ascontiguousarray(scales, np.float32)
            tptr, sptr = _p(self.table).value, _p(self.scales).value
        else:
            self._lh = _LobesHold(lobes)
            lptr = C.cast(C.pointer(self._lh.s), C.c_void_p).value
        self.s = _Scene(self.R, (C.c_double * 3)(*self.O), M, N, Cc, K, _p(self.Po).value,
                        _p(self.Pd).value, dt, tptr, sptr, lptr, rptr, 1 if upper else 0)


def _views_arrays(views):
    vf = np.ascontiguousarray(np.stack([v.floats14() for v in views]), np.float32)
    wh = np.ascontiguousarray(np.array([[v.width, v.height] for v in views], np.uint32))
    return vf, wh


def render_pixels(scene: Scene, views, pix: np.ndarray, threads: Optional[int] = None):
    """Render pixels pix [n,3] = (view, x, y): (out [n,C] FP64, idx [n,2K], hits)."""
    pix = np.ascontiguousarray(pix, np.uint32)
    n = pix.shape[0]
    vf, wh = _views_arrays(views)
    out = np.zeros((n, scene.C))
    idx = np.zeros((n, 2 * scene.K), np.int32)
    L = lib()
    nt = min(_threads(threads), max(1, n // 64))
    bounds = np.linspace(0, n, nt * 4 + 1).astype(np.int64)

    def work(k):
        a, b = int(bounds[k]), int(bounds[k + 1])
        if b <= a:
            return 0
        return L.lfo_render_pixels(C.byref(scene.s), _p(vf), _p(wh), _p(pix[a:]), b - a,
                                   _p(out[a:]), _p(idx[a:]))
    with ThreadPoolExecutor(nt) as ex:
        hits = sum(ex.map(work, range(len(bounds) - 1)))
    return out, idx, int(hits)


def render_views(scene: Scene, views, threads: Optional[int] = None):
    """Render every pixel of every view into an output buffer of
    max(out_offset + W*H) pixels: (out [P,C] FP64, idx [P,2K], hits)."""
    import lf_inputs
    P = lf_inputs.total_pixels(views)
    out = np.zeros((P, scene.C))
    idx = np.full((P, 2 * scene.K), -1, np.int32)
    pix = lf_inputs.pixel_list(views)
    o, i, hits = render_pixels(scene, views, pix, threads)
    offs = lf_inputs.pixel_offsets(views, pix)
    out[offs] = o
    idx[offs] = i
    return out, idx, hits


def render_backward(scene: Scene, views, pix: np.ndarray, grad_out: np.ndarray) -> np.ndarray:
    """G = A^T g for the blend A over pixels pix; grad_out [n,C]; G [M,N,C] FP64."""
    pix = np.ascontiguousarray(pix, np.uint32)
    g = np.ascontiguousarray(grad_out, np.float64).reshape(pix.shape[0], scene.C)
    vf, wh = _views_arrays(views)
    G = np.zeros((scene.M // 2 if scene.s.upper else scene.M, scene.N, scene.C))
    lib().lfo_render_backward_pixels(C.byref(scene.s), _p(vf), _p(wh), _p(pix), pix.shape[0],
                                     _p(g), _p(G))
    return G


def psnr(ref: np.ndarray, test: np.ndarray, hit: np.ndarray) -> float:
    """10 log10(peak^2 / MSE) over hit pixels and all channels; peak = max of ref
    over those entries."""
    ref = np.asarray(ref, np.float64)[hit]
    test = np.asarray(test, np.float64)[hit]
    if ref.size == 0:
        return float("nan")
    mse = float(np.mean((ref - test) ** 2))
    peak = float(ref.max())
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)
