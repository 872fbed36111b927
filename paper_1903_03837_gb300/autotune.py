"""Launch-shape autotuner for the render kernel.

Times candidate launch shapes (CTA tile, warp sub-tile, tile order, static or
persistent grid) on the caller's own views with CUDA events and keeps the
fastest. Results are cached per (key, device name) in a JSON file next to the
built library, so a workload is tuned once per machine.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, List, Sequence

from . import build as _build

CACHE = os.path.join(_build.BUILD, "autotune.json")
_lock = threading.Lock()

# (tile_w, tile_h, warp_w, order, persistent)
CANDIDATES = [
    (16, 16, 8, 0, 0), (16, 16, 8, 1, 0), (16, 16, 8, 0, 1), (16, 16, 8, 1, 1),
    (32, 8, 8, 0, 0), (32, 8, 8, 1, 1), (8, 32, 8, 0, 0), (16, 8, 8, 0, 0),
    (16, 16, 16, 0, 0), (32, 8, 32, 0, 0), (16, 16, 4, 0, 0), (64, 4, 8, 1, 1),
    (32, 4, 8, 0, 0), (8, 16, 8, 1, 1), (16, 8, 4, 0, 0),
]
QUICK = [(16, 16, 8, 0, 0), (16, 16, 8, 1, 1), (32, 8, 8, 0, 0), (16, 8, 8, 0, 0)]


def as_launch(c) -> Dict[str, int]:
    return dict(tile_w=c[0], tile_h=c[1], warp_w=c[2], order=c[3], persistent=c[4], ctas_per_sm=0)


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_launch(lf, view_sets: Sequence[Sequence], launch: Dict[str, int], reps: int = 3) -> float:
    """Mean ms per view set for one launch shape (after one untimed pass)."""
    import torch
    lf.set_launch(**launch)
    outs = [torch.empty((max(int(v.out_offset) + v.width * v.height for v in vs), lf.C),
                        dtype=torch.float32, device="cuda") for vs in view_sets]
    for vs, o in zip(view_sets, outs):
        lf.render(vs, out=o)
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        for vs, o in zip(view_sets, outs):
            lf.render(vs, out=o)
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / (reps * len(view_sets))


def tune(lf, view_sets: Sequence[Sequence], candidates=None, reps: int = 3) -> List[tuple]:
    """[(ms, launch)] for every candidate, fastest first."""
    res = []
    for c in (candidates or CANDIDATES):
        L = as_launch(c)
        res.append((time_launch(lf, view_sets, L, reps), L))
    res.sort(key=lambda r: r[0])
    return res


def best_launch(lf, view_sets: Sequence[Sequence], key: str, quick: bool = False,
                retune: bool = False) -> Dict[str, int]:
    """Cached best launch shape for `key` on this device (tuned on first use)."""
    import torch
    dev = torch.cuda.get_device_name()
    ck = f"{key}|{dev}|{lf.dtype}|{lf.M}x{lf.N}"
    with _lock:
        cache = _load()
        if not retune and ck in cache:
            lf.set_launch(**cache[ck]["launch"])
            return cache[ck]["launch"]
        res = tune(lf, view_sets, QUICK if quick else CANDIDATES)
        best = res[0][1]
        cache[ck] = {"launch": best, "ms": res[0][0],
                     "all": [[round(ms, 4), L] for ms, L in res]}
        _store(cache)
    lf.set_launch(**best)
    return best
