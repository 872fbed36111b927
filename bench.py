"""Benchmark of the light-field sampling path on the large workload.

Workload: 262,144 origin x 4,096 direction SF points, RGBA lobe-field table
stored as E4M3 (4 GiB, headline), FP16 (8 GiB) and FP32 (16 GiB) with per-row
FP32 scales; a 240-frame orbit at 3R, each frame a 3840x2160 stereo pair
(16,588,800 rays) rendered in one launch. A step renders one frame.

Prints one JSON line: Grays/s over all pixels (value, device-timed with CUDA
events), the end-to-end figure through the public API with the image read
back to pinned host memory every step (e2e), the roofline of the render
kernel against the measured HBM copy bandwidth, the SM clocks seen during the
timed region, and the CPU oracle timed on a bounded sample (cpu_baseline).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
Multi-GPU (torchrun): every rank renders its own frames (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lf_inputs  # noqa: E402

METRIC = "Grays/s light-field lookup (FP16/FP8 vs FP32 table at stated PSNR); % HBM peak"
UNIT = "Grays/s"
TEXEL_BYTES = {"f32": 16, "f16": 8, "e4m3": 4}
SCALE_BYTES = {"f32": 0, "f16": 20, "e4m3": 20}
OUT_BYTES = 16


def workload_name(cfg) -> str:
    return (f"large: {cfg.M:,} x {cfg.N:,} RGBA lobe-field table (E4M3 4 GiB headline; FP16 8 GiB, "
            f"FP32 16 GiB variants) with per-row FP32 scales; 240-frame orbit at 3R, elevation 20 deg, "
            f"one 3840x2160 stereo pair per frame ({cfg.rays:,} rays) in one launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


RENDER_SOURCES = ("paper_1903_03837_gb300/csrc/lf_render.cu", "paper_1903_03837_gb300/csrc/lf_device.cuh",
                  "paper_1903_03837_gb300/csrc/lf_kernels.h", "paper_1903_03837_gb300/csrc/lf_internal.h",
                  "include/lumipath.h", "paper_1903_03837_gb300/build.py")


def csrc_digest() -> str:
    """SHA-256 over the files the render kernel is compiled from: its
    translation unit and the headers it includes, and the build script that
    holds the compiler flags (name + content, in this order)."""
    import hashlib
    h = hashlib.sha256()
    for n in RENDER_SOURCES:
        h.update(n.encode())
        with open(os.path.join(ROOT, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


_WORKLOAD = {"name": "large"}


def _recorded():
    """The per-launch counters of the render kernel on the large workload from the
    ncu launch list summarised in profiles/render_traffic.txt; {} when the kernel
    sources have changed since that capture, or for another workload."""
    p = os.path.join(ROOT, "profiles", "render_traffic.txt")
    if not os.path.exists(p) or _WORKLOAD["name"] != "large":
        return {}
    rec = {}
    with open(p) as f:
        for ln in f:
            parts = ln.split()
            if len(parts) == 2 and not ln.startswith("#"):
                rec[parts[0]] = parts[1]
    return rec if rec.get("csrc_sha256") == csrc_digest() else {}


def recorded_counter(dtype: str, name: str):
    """A recorded per-launch counter (see _recorded), or None."""
    v = _recorded().get(f"{dtype}_{name}")
    return int(v) if v else None


def recorded_pct(dtype: str, name: str):
    """A recorded percentage of peak (ncu, the capture's own launch time), or None."""
    v = _recorded().get(f"{dtype}_{name}")
    return float(v) if v else None


def recorded_traffic(dtype: str):
    """DRAM bytes (read + write) per launch, or None (see _recorded)."""
    return recorded_counter(dtype, "dram_bytes_per_launch")


def compulsory_bytes(idx_hit, N: int, rays: int, dtype: str) -> dict:
    """Compulsory DRAM bytes of one frame: the image (16 B per ray) plus the
    distinct 32-byte sectors of texels and of row scales that its 25 taps per hit
    ray touch (idx_hit: int32 [hits, 10], 5 origin then 5 direction indices)."""
    import torch
    tb = TEXEL_BYTES[dtype]
    io, jd = idx_hit[:, :5].long(), idx_hit[:, 5:].long()
    ok = (io >= 0).unsqueeze(2) & (jd >= 0).unsqueeze(1)
    tex = (io.unsqueeze(2) * N + jd.unsqueeze(1))[ok]
    tex_sectors = int(torch.unique((tex * tb) // 32).numel())
    scale_sectors = int(torch.unique((io[io >= 0] * 4) // 32).numel()) if dtype != "f32" else 0
    return {"bytes": rays * 16 + 32 * (tex_sectors + scale_sectors), "image_bytes": rays * 16,
            "texel_sectors": tex_sectors, "scale_sectors": scale_sectors}


def issue_roofline(dtype: str, launch_s: float):
    """The render kernel against the SM issue rate (it is issue-bound): thread
    instructions per launch (recorded by ncu) / the live launch time, against
    SMs x 4 schedulers x 32 lanes x the maximum SM clock; None without a record."""
    v = _recorded().get(f"{dtype}_thread_inst_per_launch")
    if not v:
        return None
    from paper_1903_03837_gb300 import lumipath as lp
    sms, mhz = lp.lf_device_sm_count(), sm_max_mhz()
    peak = sms * 4 * 32 * mhz * 1e6 / 1e12
    achieved = int(v) / launch_s / 1e12
    return {"achieved": achieved, "peak": peak, "unit": "T thread-instructions/s", "frac": achieved / peak,
            "thread_inst_per_launch": int(v),
            "peak_source": f"derived: {sms} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        time.sleep(0.2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def algorithmic_bytes(hits: int, rays: int, dtype: str) -> int:
    return hits * (25 * TEXEL_BYTES[dtype] + SCALE_BYTES[dtype] + OUT_BYTES) + (rays - hits) * OUT_BYTES


def run_ours(args, rank: int, world: int):
    import torch
    from paper_1903_03837_gb300 import torch_api as api
    from paper_1903_03837_gb300 import lumipath as lp
    from paper_1903_03837_gb300 import autotune, replicas

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev_index = torch.cuda.current_device()
    cfg = lf_inputs.config_large() if args.workload == "large" else lf_inputs.config_precision()
    _WORKLOAD["name"] = args.workload
    lob = cfg.lobes()
    M, N = cfg.M, cfg.N
    t0 = time.time()
    T32 = api.fill_lobe_table(lob, M, N)
    tables = {"f32": api.LightField(T32, "f32", borrow=True)}
    codes = {}
    for dt in ("f16", "e4m3"):
        c, s = api.quantize_table(T32, dt)
        codes[dt] = (c, s)
        tables[dt] = api.LightField(c, dt, s, borrow=True)
    torch.cuda.synchronize()
    setup_s = time.time() - t0

    if args.workload == "large":
        frames_total = cfg.extra["frames"]
        my_frames = replicas.frames_for_rank(rank, world, args.steps + args.warmup, frames_total)
        frame_views = {f: lf_inputs.orbit_frame(f) for f in set(my_frames)}
    else:
        my_frames = [0] * (args.steps + args.warmup)
        frame_views = {0: cfg.views}
    rays = cfg.rays
    if args.launch:
        tw, th, ww, order, pers = (int(x) for x in args.launch.split(","))
        launch = dict(tile_w=tw, tile_h=th, warp_w=ww, order=order, persistent=pers, ctas_per_sm=0)
    else:
        launch = autotune.best_launch(tables[args.dtype], [frame_views[my_frames[0]]],
                                      key=f"{args.workload}-{args.dtype}", quick=args.quick_tune)
    for t in tables.values():
        t.set_launch(**launch)

    # hits per frame (untimed): from the index output; and, for the first timed
    # frame, the compulsory DRAM bytes: the image plus every distinct 32-byte
    # sector of texels and row scales the frame reads, each counted once
    hits = {}
    compulsory = None
    idx_buf = torch.empty((rays, 10), dtype=torch.int32, device="cuda")
    for f, vs in frame_views.items():
        _, idx = tables["e4m3"].render(vs, with_idx=True, idx=idx_buf)
        hit_rows = idx[:, 0] >= 0
        hits[f] = int(hit_rows.sum())
        if compulsory is None and f == my_frames[args.warmup]:
            compulsory = compulsory_bytes(idx[hit_rows], N, rays, args.dtype)
        del hit_rows
    del idx_buf, idx
    torch.cuda.empty_cache()

    outs = [torch.empty((rays, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    stream = torch.cuda.current_stream()

    def timed(dtype):
        lf = tables[dtype]
        for k in range(args.warmup):
            lf.render(frame_views[my_frames[k]], out=outs[k % 2])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for k in range(args.steps):
            f = my_frames[args.warmup + k]
            lf.render(frame_views[f], out=outs[k % 2])
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        if world > 1:
            total_ms = replicas.reduce_max(total_ms)
            torch.distributed.barrier()
        nbytes = sum(algorithmic_bytes(hits[my_frames[args.warmup + k]], rays, dtype) for k in range(args.steps))
        return total_ms, per, nbytes

    with ClockSampler(dev_index) as clk:
        total_ms, per_ms, nbytes = timed(args.dtype)
    clocks = clk.summary()
    # hit rays of the timed frames (the same frames for every table type and K)
    step_hits = sum(hits[my_frames[args.warmup + k]] for k in range(args.steps))
    variants = {}
    for dt in (("f16", "f32") if not args.no_variants else ()):
        if dt == args.dtype:
            continue
        # each table type at its own best launch shape (the 16-byte FP32 texels
        # favour narrower warp tiles than the 4-byte E4M3 ones)
        vlaunch = launch if args.launch else autotune.best_launch(
            tables[dt], [frame_views[my_frames[0]]], key=f"{args.workload}-{dt}", quick=args.quick_tune)
        tm, pm, nb = timed(dt)
        variants[dt] = {"grays_s": world * args.steps * rays / (tm * 1e-3) / 1e9,
                        "hit_grays_s": world * step_hits / (tm * 1e-3) / 1e9,
                        "ms_per_step": tm / args.steps, "launch": vlaunch,
                        "hbm_frac_of_measured": nb / (sum(pm) * 1e-3) / 1e9 / measured_peaks()[0]}

    # quality of the quantised tables against the FP32-table image (full frame, GPU)
    f0 = my_frames[0]
    ref, idx = tables["f32"].render(frame_views[f0], with_idx=True)
    hitmask = idx[:, 0] >= 0
    psnr_vs_f32 = {}
    for dt in ("f16", "e4m3"):
        img, _ = tables[dt].render(frame_views[f0])
        r, g = ref[hitmask].double(), img[hitmask].double()
        mse = float(((r - g) ** 2).mean())
        psnr_vs_f32[dt] = 10 * math.log10(float(r.max()) ** 2 / mse) if mse > 0 else float("inf")
    gpu_images = {dt: tables[dt].render(frame_views[f0])[0] for dt in ("f32", "f16", "e4m3")}

    # Neighbour count (Section 2: nearest sampling, five, "up to nine"): the same
    # frames and launch shape on the headline table with K = 1 and K = 9, and the
    # FP32-table image of each K for the quality comparison of the CPU leg.
    neighbours = {5: {"grays_s": world * args.steps * rays / (total_ms * 1e-3) / 1e9,
                      "hit_grays_s": world * step_hits / (total_ms * 1e-3) / 1e9,
                      "ms_per_step": total_ms / args.steps}}
    k_images = {5: gpu_images["f32"]}
    if not args.no_variants and args.workload == "large":
        for K in (1, 9):
            c, sc = codes[args.dtype] if args.dtype != "f32" else (T32, None)
            lfk = api.LightField(c, args.dtype, sc, borrow=True, k_nearest=K)
            lfk.set_launch(**launch)
            for k in range(3):
                lfk.render(frame_views[my_frames[k]], out=outs[k % 2])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                lfk.render(frame_views[my_frames[args.warmup + k]], out=outs[k % 2])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            neighbours[K] = {"grays_s": world * rays / (ms * 1e-3) / 1e9,
                             "hit_grays_s": world * step_hits / args.steps / (ms * 1e-3) / 1e9, "ms_per_step": ms}
            lfk.close()
            lf32 = api.LightField(T32, "f32", borrow=True, k_nearest=K)
            lf32.set_launch(**launch)
            k_images[K] = lf32.render(frame_views[f0])[0]
            torch.cuda.synchronize()
            lf32.close()

    # End to end through the public API: the host views go in with each call and
    # every frame's image is read back to pinned host memory. Double-buffered:
    # frame k+1 renders on the compute stream while frame k copies on a second one.
    lf = tables[args.dtype]
    copy_stream = torch.cuda.Stream()

    def e2e_run(half: bool):
        """Three timed windows of K frames each, double-buffered; returns the
        window times (the median is reported: the device-to-host copies share
        the host's memory system with other work)."""
        odt = torch.float16 if half else torch.float32
        dev = outs if not half else [torch.empty((rays, 4), dtype=odt, device="cuda") for _ in range(2)]
        host = [torch.empty((rays, 4), dtype=odt, pin_memory=True) for _ in range(2)]
        rendered = [torch.cuda.Event() for _ in range(2)]
        copied = [torch.cuda.Event() for _ in range(2)]

        def e2e_frame(k, f):
            b = k % 2
            stream.wait_event(copied[b])
            lf.render(frame_views[f], out=dev[b], half=half)
            rendered[b].record(stream)
            copy_stream.wait_event(rendered[b])
            with torch.cuda.stream(copy_stream):
                host[b].copy_(dev[b], non_blocking=True)
                copied[b].record(copy_stream)
        for k in range(2):
            copied[k].record(copy_stream)
        for k in range(min(3, args.warmup)):
            e2e_frame(k, my_frames[k])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wins = []
        for _ in range(3):
            t_e2e = time.perf_counter()
            for k in range(args.steps):
                e2e_frame(k, my_frames[args.warmup + k])
            torch.cuda.synchronize()
            w_s = time.perf_counter() - t_e2e
            if world > 1:
                w_s = replicas.reduce_max(w_s)
            wins.append(w_s)
        return wins, host

    e2e_windows, host = e2e_run(False)
    e2e_s = sorted(e2e_windows)[1]
    # The link's ceiling for this metric: the same device-to-host copy alone
    # (median of three groups of 5 copies, right after the timed windows).
    cp = []
    for _ in range(3):
        torch.cuda.synchronize()
        t_cp = time.perf_counter()
        for k in range(5):
            host[k % 2].copy_(outs[k % 2], non_blocking=True)
        torch.cuda.synchronize()
        cp.append(5 * rays * 16 / (time.perf_counter() - t_cp) / 1e9)
    d2h_gbs = sorted(cp)[1]
    e2e16_windows, _ = e2e_run(True)
    e2e16_s = sorted(e2e16_windows)[1]

    peak, peak_kind = measured_peaks()
    avg_launch_s = sum(per_ms) / len(per_ms) * 1e-3
    bytes_per_launch = nbytes / args.steps
    achieved = bytes_per_launch / avg_launch_s / 1e9
    value = world * args.steps * rays / (total_ms * 1e-3) / 1e9
    hit_frac = float(np.mean([hits[f] for f in my_frames[args.warmup:]]) / rays)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT,
        "hit_grays_s": world * step_hits / (total_ms * 1e-3) / 1e9, "hit_fraction": hit_frac,
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(cfg) if args.workload == "large" else
                   f"precision: {cfg.M:,} x {cfg.N:,} RGBA table, one 1920x1080 view at 2.5R",
                   "table_storage": args.dtype,
                   "rays_per_step": rays, "hit_fraction": hit_frac,
                   "l2": "inputs larger than L2: 4 GiB table, 265 MB image per step, orbit frame changes every step",
                   "launch": launch, "parallelism": f"replicas x{world} (views sharded, no collective)",
                   "setup_s": round(setup_s, 2)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(args.dtype),
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "kernel": f"lfk::render_kernel<{args.dtype}> with the lfk::fixup_kernel that follows it "
                               f"(the exact pass of the rays left uncertain); timed together, per step",
                     "avg_launch_ms": avg_launch_s * 1e3,
                     "compulsory_bytes_per_launch": compulsory["bytes"] if compulsory else None,
                     "l2_bytes_per_launch": recorded_counter(args.dtype, "l2_bytes_per_launch"),
                     "l2_achieved_gbs": (recorded_counter(args.dtype, "l2_bytes_per_launch") or 0) / avg_launch_s / 1e9
                     or None,
                     "l2_pct_of_peak_ncu": recorded_pct(args.dtype, "l2_pct_of_peak"),
                     "dram_pct_of_peak_ncu": recorded_pct(args.dtype, "dram_pct_of_peak"),
                     "issue": issue_roofline(args.dtype, avg_launch_s)},
        "clocks": clocks,
        "e2e": {"value": world * args.steps * rays / e2e_s / 1e9, "unit": UNIT,
                "hit_grays_s": world * step_hits / e2e_s / 1e9,
                "h2d_bytes_per_step": 2 * 72, "d2h_bytes_per_step": rays * 16,
                "how": "lf_render per frame with host lf_view structs, image copied to pinned host "
                       "memory every frame on a second stream (double-buffered); median of 3 "
                       "windows of K frames",
                "windows_grays_s": [world * args.steps * rays / w / 1e9 for w in e2e_windows],
                "d2h_copy_gbs": d2h_gbs, "copy_bound_grays_s": world * d2h_gbs / 16.0,
                "binary16_image": {"value": world * args.steps * rays / e2e16_s / 1e9, "unit": UNIT,
                                   "d2h_bytes_per_step": rays * 8,
                                   "how": "the same loop through lf_render_f16 (each value of the FP32 "
                                          "image rounded once to binary16), median of 3 windows"}},
        "gpu_launches": 2 * args.steps,      # render kernel + fixup kernel per step
        "variants": variants,
        "psnr_vs_f32_table_db": psnr_vs_f32,
        "neighbours": {str(k): v for k, v in sorted(neighbours.items())},
    }
    if not args.no_variants:
        for t in tables.values():
            t.close()
        del T32, codes, tables, outs
        torch.cuda.empty_cache()
        line["fit"] = run_fit_steps(args)
        torch.cuda.empty_cache()
        line["paper_shape"] = run_paper_shape(args)
        torch.cuda.empty_cache()
        line["batching"] = run_batching(args)
        torch.cuda.empty_cache()
        line["precompute"] = run_precompute(args)
        torch.cuda.empty_cache()
        line["post_filter"] = run_post_filter(args)
        tables = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "large":
        line["cpu_baseline"], psnr64, psnr_k = cpu_baseline(cfg, frame_views[f0], gpu_images, args, k_images)
        line["psnr_vs_fp64_db"] = psnr64
        for k, v in psnr_k.items():
            line["neighbours"][str(k)]["psnr_vs_continuous_field_db"] = v
    for t in tables.values():
        t.close()
    return line


def sm_max_mhz() -> float:
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", os.environ.get("LOCAL_RANK", "0")], capture_output=True, text=True,
                             timeout=20).stdout.split()
        return float(out[0])
    except Exception:
        return 2070.0


def run_precompute(args):
    """Light-field precompute (Section 2) of the analytic volume scene into a
    16,384 x 512 RGBA FP32 table: 8 blobs, 4 jittered samples per texel, 64
    midpoint steps. ALU-bound: the roofline counts the algorithm's FP32 lane
    operations per midpoint step -- per blob, 2 for the blob's exponent (a
    quadratic in t), 1 to add its density and 1 to add its weighted emission;
    10 per step for the step's weight and transmittance -- against the FP32
    issue rate (SMs x 128 lanes x max SM clock), and its exp2 evaluations (one
    per blob-step plus one per step) against 32 per SM per clock (the XU rate
    this GPU showed: 28.5% XU utilisation at 2.54 T exp2/s)."""
    import torch
    from paper_1903_03837_gb300 import torch_api as api
    from paper_1903_03837_gb300 import lumipath as lp
    cfg = lf_inputs.config_precompute()
    vol = cfg.extra["volume"]
    M, N, C = cfg.M, cfg.N, cfg.C
    out = torch.empty((M, N, C), dtype=torch.float32, device="cuda")
    for _ in range(3):
        api.precompute_table(vol, M, N, C, out=out)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    reps = max(3, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        api.precompute_table(vol, M, N, C, out=out)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    texels = M * N
    samples = texels * vol.spp
    steps = samples * vol.steps
    fp32_ops = steps * (4 * vol.B + 10)
    exp2s = steps * (vol.B + 1)
    sms, mhz = lp.lf_device_sm_count(), sm_max_mhz()
    fp32_peak = sms * 128 * mhz * 1e6 / 1e12
    xu_peak = sms * 32 * mhz * 1e6 / 1e12
    achieved = fp32_ops / (ms * 1e-3) / 1e12
    versus = light_field_vs_direct(args, vol, cfg.views, out)
    del out
    return {"workload": f"precompute: {M:,} x {N:,} RGBA FP32 table of a {vol.B}-blob emission-absorption "
                        f"volume, {vol.spp} jittered samples per texel, {vol.steps} midpoint steps",
            "ms_per_table": ms, "gtexels_s": texels / (ms * 1e-3) / 1e9,
            "gsamples_s": samples / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / fp32_peak,
                         "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz",
                         "exp2_per_s_T": exp2s / (ms * 1e-3) / 1e12,
                         "exp2_frac_of_32_per_sm_clk": exp2s / (ms * 1e-3) / 1e12 / xu_peak,
                         "kernel": "lfk::precompute_kernel<8>"},
            "light_field_vs_direct": versus}


def light_field_vs_direct(args, vol, views, table):
    """The light field against the scene itself: the direct render of the
    volume along every pixel's ray (lf_render_volume, the ground truth) and the
    light-field render of the precomputed table for the same views, both timed
    with CUDA events, and the PSNR of the light-field image against the direct
    one over the hit pixels -- for the given table and for a larger one."""
    import torch
    from paper_1903_03837_gb300 import torch_api as api
    st = torch.cuda.current_stream()
    rays = lf_inputs.total_pixels(views)
    reps = max(3, min(args.steps, 10))

    def timed(fn):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    gt = torch.empty((rays, 4), device="cuda")
    direct_ms = timed(lambda: api.render_volume(vol, views, 4, out=gt))
    gt_np = gt.cpu().numpy()
    img = torch.empty((rays, 4), device="cuda")
    res = {"views": f"{len(views)} views, {rays:,} rays", "steps": vol.steps,
           "direct_ms": direct_ms, "direct_grays_s": rays / (direct_ms * 1e-3) / 1e9, "tables": {}}
    M0, N0 = int(table.shape[0]), int(table.shape[1])
    for M, N in ((M0, N0), (4 * M0, 4 * N0)):
        T = table if (M, N) == (M0, N0) else api.precompute_table(vol, M, N, 4)
        lf = api.LightField(T, "f32", borrow=True)
        lf.set_launch(tile_w=16, tile_h=8, warp_w=8)
        _, idx = lf.render(views, out=img, with_idx=True)
        hit = idx[:, 0].cpu().numpy() >= 0
        ms = timed(lambda: lf.render(views, out=img))
        img_np = img.cpu().numpy()
        ssim = [ssim_mean(gt_np[v.out_offset:v.out_offset + v.pixels, :3].reshape(v.height, v.width, 3),
                          img_np[v.out_offset:v.out_offset + v.pixels, :3].reshape(v.height, v.width, 3),
                          hit[v.out_offset:v.out_offset + v.pixels].reshape(v.height, v.width),
                          float(gt_np[hit, :3].max()))
                for v in views]
        res["tables"][f"{M:,} x {N:,}"] = {
            "light_field_ms": ms, "light_field_grays_s": rays / (ms * 1e-3) / 1e9,
            "psnr_vs_direct_db": psnr_db(gt_np[:, :3], img_np[:, :3], hit),
            "ssim_vs_direct": float(np.mean(ssim)),
            "hit_fraction": float(hit.mean())}
        lf.close()
        del T
    return res


def psnr_db(ref, test, hit):
    """10 log10(peak^2 / MSE) over the hit pixels' channels, peak = max of ref there."""
    r = np.asarray(ref, np.float64)[hit]
    t = np.asarray(test, np.float64)[hit]
    mse = float(np.mean((r - t) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(float(r.max()) ** 2 / mse)


def run_post_filter(args):
    """Learned post-filter (Section 2, post-processing; the generator's loss,
    no adversary): trained on the light-field renders of 40 volume scenes'
    1,024 x 256 tables against their direct renders, then measured on 8
    held-out scenes (4 views of 256x256 each): PSNR and SSIM against the direct
    render before and after the filter (lf_post_filter), next to a 16x larger
    table without it, and the filter's time per frame next to the render's."""
    import torch
    from paper_1903_03837_gb300 import torch_api as api, post_filter as pf
    cfg = lf_inputs.config_post_filter()
    M, N = cfg.M, cfg.N
    t0 = time.time()
    feats, targets, _ = pf.make_pairs(cfg.extra["train"], M, N)
    t1 = time.time()
    steps = 2000
    w, hist = pf.train(feats, targets, steps=steps, batch=16)
    torch.cuda.synchronize()
    t2 = time.time()
    del feats, targets
    st = torch.cuda.current_stream()
    reps = max(3, min(args.steps, 10))

    def timed(fn):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = {"light_field": [], "filtered": [], "light_field_16x": []}
    ssims = {k: [] for k in rows}
    filt = pf.PostFilter(w)
    for vol, views in cfg.extra["test"]:
        gt = api.render_volume(vol, views, 4)
        gt_np = gt.cpu().numpy()
        out = {}
        for key, (m, n) in (("light_field", (M, N)), ("light_field_16x", (4 * M, 4 * N))):
            T = api.precompute_table(vol, m, n, 4)
            lf = api.LightField(T, "f32", borrow=True)
            img, idx = lf.render(views, with_idx=True)
            if key == "light_field":
                out["filtered"] = filt(views, img).cpu().numpy()
                hit = idx[:, 0].cpu().numpy() >= 0
            out[key] = img.cpu().numpy()
            lf.close()
            del T
        peak = float(gt_np[hit, :3].max())
        for key, im in out.items():
            rows[key].append((gt_np[hit, :3], im[hit, :3], peak))
            for v in views:
                a, b = v.out_offset, v.out_offset + v.pixels
                ssims[key].append(ssim_mean(gt_np[a:b, :3].reshape(v.height, v.width, 3),
                                            im[a:b, :3].reshape(v.height, v.width, 3),
                                            hit[a:b].reshape(v.height, v.width), peak))

    def psnr_all(rs):
        mse = np.mean(np.concatenate([((r - t) ** 2).ravel() for r, t, _ in rs]))
        peak = max(p for _, _, p in rs)
        return 10.0 * math.log10(peak * peak / mse)
    # time per frame: one 1920x1080 view of the first held-out scene, rendered
    # from its table and filtered
    vol = cfg.extra["test"][0][0]
    frame = [lf_inputs.look_at((2.2, -1.1, 0.9), (0, 0, 0), 1920, 1080)]
    T = api.precompute_table(vol, M, N, 4)
    lf = api.LightField(T, "f32", borrow=True)
    img, _ = lf.render(frame)
    render_ms = timed(lambda: lf.render(frame, out=img))
    filtered = filt(frame, img)
    filt_ms = timed(lambda: filt(frame, img, out=filtered))
    lf.close()
    del T
    px = 1920 * 1080
    n_scenes = len(cfg.extra["test"])
    return {"workload": f"post-filter: trained on {len(cfg.extra['train'])} volume scenes x 8 views 128x128, "
                        f"tested on {n_scenes} held-out scenes x 4 views 256x256; {M:,} x {N:,} RGBA FP32 tables",
            "train_steps": steps, "train_s": round(t2 - t1, 2), "data_s": round(t1 - t0, 2),
            "loss_first_last": [hist[0], hist[-1]],
            "psnr_vs_direct_db": {k: psnr_all(v) for k, v in rows.items()},
            "ssim_vs_direct": {k: float(np.mean(v)) for k, v in ssims.items()},
            "frame": "1920x1080", "filter_ms_per_frame": filt_ms, "render_ms_per_frame": render_ms,
            "filter_gpixels_s": px / (filt_ms * 1e-3) / 1e9,
            "filter_tflops": 2 * px * (4 * 16 * 9 + 16 * 16 * 9 + 16 * 3 * 9) / (filt_ms * 1e-3) / 1e12,
            "kernel": "lfk::post_filter_kernel (all three layers tcgen05.mma kind::f16, M = 128 positions x "
                      "N = 48 (16 channels x 3 output rows) x K = 16, FP16 operands in shared memory, FP32 "
                      "accumulators in tensor memory; a 124-column strip per CTA in bands of 6 rows, 2 CTAs per SM)"}


def ssim_mean(ref, img, mask, data_range):
    """Mean structural similarity (Wang et al., 2004: Gaussian window of standard
    deviation 1.5 truncated to 11 x 11, C1 = (0.01 L)^2, C2 = (0.03 L)^2) of one
    view's image [H, W, C] against the reference, averaged over the channels and
    over the pixels of `mask` [H, W] -- the quality measure the paper reports
    against its path-traced ground truth (Section 3)."""
    from scipy.ndimage import gaussian_filter
    x = np.asarray(ref, np.float64)
    y = np.asarray(img, np.float64)
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    g = lambda a: gaussian_filter(a, sigma=1.5, truncate=3.5, mode="nearest")
    maps = []
    for c in range(x.shape[2]):
        a, b = x[:, :, c], y[:, :, c]
        mx, my = g(a), g(b)
        vx = g(a * a) - mx * mx
        vy = g(b * b) - my * my
        cxy = g(a * b) - mx * my
        maps.append(((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2)))
    return float(np.mean(np.mean(maps, axis=0)[mask]))


def run_fit_steps(args):
    """Differentiation workload: 16,384 x 512 RGB FP32 table, 32 target views of
    512x512 per rank (weak scaling: rank r fits views 32r .. 32r+31 of one
    seeded pool); one step = render (forward kernel, writing its sample indices)
    + MSE + backward scatter kernel from those indices + one all-reduce of the
    gradient table over the ranks + Adam on the FP32 table (torch_api.fit_step).
    Times the steps and the backward launches alone, and once more the backward
    that searches the indices again (lf_render_backward)."""
    import torch
    from paper_1903_03837_gb300 import replicas
    from paper_1903_03837_gb300 import torch_api as api
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    base = lf_inputs.config_differentiation()
    n_train = base.extra["n_train"]
    cfg = lf_inputs.config_differentiation(n_train=n_train * world)
    train = lf_inputs.pack_offsets(replicas.shard(cfg.views[:n_train * world], rank, world))
    rays = lf_inputs.total_pixels(train)
    gt = api.fill_lobe_table(cfg.lobes(), cfg.M, cfg.N)
    lf_gt = api.LightField(gt, "f32", borrow=True)
    target, _ = lf_gt.render(train)
    table = torch.zeros_like(gt, requires_grad=True)
    table.grad = torch.zeros_like(table)
    lf = api.LightField(table.detach(), "f32", borrow=True)
    # the default (multi-tensor) Adam: 0.29 ms per step here, the fused one measured 1.11 ms
    opt = torch.optim.Adam([table], lr=cfg.extra["lr"], betas=(0.9, 0.999), eps=1e-8)
    st = torch.cuda.current_stream()
    idx = torch.empty((rays, 2 * lf.K), dtype=torch.int32, device="cuda")
    global_values = rays * world * cfg.C
    for _ in range(args.warmup):
        api.fit_step(lf, table, opt, train, target, idx, global_values)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        api.fit_step(lf, table, opt, train, target, idx, global_values)
    e1.record(st)
    torch.cuda.synchronize()
    ms = replicas.reduce_max(e0.elapsed_time(e1) / args.steps)
    # the backward alone: from the forward's indices, and searching again
    g = (2.0 / global_values) * (lf.render(train, idx=idx)[0] - target)
    res = {}
    for name, kw in (("backward_ms", {"idx": idx}), ("backward_search_ms", {})):
        for _ in range(2):
            lf.render_backward(train, g, table.grad, **kw)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(5):
            lf.render_backward(train, g, table.grad, **kw)
        b.record(st)
        torch.cuda.synchronize()
        res[name] = replicas.reduce_max(a.elapsed_time(b) / 5)
    lf.close()
    lf_gt.close()
    bms = res["backward_ms"]
    return {"workload": f"differentiation: {cfg.M:,} x {cfg.N:,} RGB FP32 table, {len(train)} views 512x512 "
                        f"per rank ({rays:,} rays per rank), Adam lr 1e-2, gradient all-reduce over "
                        f"{world} rank(s)",
            "ms_per_fit_step": ms, "fit_steps_per_s": 1e3 / ms,
            "backward_ms": bms, "backward_grays_s": world * rays / (bms * 1e-3) / 1e9,
            "backward_search_ms": res["backward_search_ms"],
            "fwd_bwd_adam_grays_s": world * rays / (ms * 1e-3) / 1e9}


def run_batching(args):
    """Batching workload: 16,384 x 512 RGBA FP16 table, 64 views of uneven size
    (16 stereo pairs of 1440x1600, 256x256, 2048x1080, 30 random multiples of 8)
    rendered in one persistent launch that a CUDA graph replays; the autotuner
    picks tile shape and ray order for the persistent grid."""
    import torch
    from paper_1903_03837_gb300 import torch_api as api, autotune
    cfg = lf_inputs.config_batching()
    T32 = api.fill_lobe_table(cfg.lobes(), cfg.M, cfg.N)
    codes, s = api.quantize_table(T32, "f16")
    del T32
    lf = api.LightField(codes, "f16", s, borrow=True)
    persistent = [c for c in autotune.CANDIDATES if c[4] == 1]
    ranked = autotune.tune(lf, [cfg.views], persistent, reps=2)
    launch = ranked[0][1]
    lf.set_launch(**launch)
    out = torch.empty((cfg.rays, 4), device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        lf.render(cfg.views, out=out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lf.render(cfg.views, out=out)
    for _ in range(args.warmup):
        graph.replay()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(args.steps):
        graph.replay()
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    lf.close()
    hit = int((out[:, 3] != 0).sum().item())      # misses store alpha 0; hits blend positive alphas
    return {"workload": f"batching: {cfg.M:,} x {cfg.N:,} RGBA FP16 table, {len(cfg.views)} views of uneven "
                        f"size ({cfg.rays:,} rays) in one persistent launch replayed from a CUDA graph",
            "launch": launch, "ms_per_batch": ms, "grays_s": cfg.rays / (ms * 1e-3) / 1e9,
            "hit_fraction": hit / cfg.rays, "hit_grays_s": hit / (ms * 1e-3) / 1e9,
            "autotune_top3_ms": [round(r[0], 4) for r in ranked[:3]]}


def run_paper_shape(args):
    """The paper's own table shape: M = 12,288 origins with only the upper
    hemisphere stored (6,144 rows), N = 23,576 directions, 4-byte E4M3 texels
    (579,403,776 bytes), rendered as a 1280x720 stereo pair per step."""
    import torch
    from paper_1903_03837_gb300 import torch_api as api
    cfg = lf_inputs.config_paper()
    rows = cfg.M // 2
    T32 = api.fill_lobe_table(cfg.lobes(), cfg.M, cfg.N)[:rows].contiguous()
    codes, s = api.quantize_table(T32, "e4m3")
    del T32
    lf = api.LightField(codes, "e4m3", s, borrow=True, n_origins=cfg.M, upper=True)
    lf.set_launch(tile_w=16, tile_h=8, warp_w=8)
    out = torch.empty((cfg.rays, 4), device="cuda")
    for _ in range(args.warmup):
        lf.render(cfg.views, out=out)
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(args.steps):
        lf.render(cfg.views, out=out)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    lf.close()
    hit = int((out[:, 3] != 0).sum().item())      # misses and masked pixels store alpha 0
    return {"workload": f"paper shape: M = {cfg.M:,} (upper {rows:,} rows stored) x N = {cfg.N:,}, "
                        f"E4M3 RGBA ({codes.numel():,} bytes), 1280x720 stereo pair ({cfg.rays:,} rays)",
            "ms_per_stereo_frame": ms, "stereo_frames_per_s": 1e3 / ms,
            "grays_s": cfg.rays / (ms * 1e-3) / 1e9, "hit_fraction": hit / cfg.rays,
            "hit_grays_s": hit / (ms * 1e-3) / 1e9,
            "paper_context": "paper: about 5.2-9.1 fps for both eyes on a HoloLens v1 (graphics-API "
                             "render, resolution not stated); other hardware, context only"}


def cpu_baseline(cfg, views, gpu_images, args, k_images=None):
    """The CPU oracle (brute-force K-NN, FP64) on a bounded random sample of the
    frame's pixels; also the FP64 reference of those pixels for PSNR, and the
    continuous lobe field along each sampled pixel's ray, the reference for the
    images of each neighbour count (FP32 table, so only interpolation differs)."""
    import oracle
    cores = host_cores()
    sc = oracle.Scene(cfg.M, cfg.N, 4, "lobe", lobes=cfg.lobes())
    oracle.sf_points(cfg.M)
    oracle.sf_points(cfg.N)
    probe = lf_inputs.sample_pixels(views, 2000, seed=11)
    t = time.perf_counter()
    oracle.render_pixels(sc, views, probe, threads=cores)
    rate = len(probe) / (time.perf_counter() - t)
    n = int(min(max(4000, rate * args.cpu_seconds), cfg.rays))
    pix = lf_inputs.sample_pixels(views, n, seed=12)
    t = time.perf_counter()
    ref, idx, hits = oracle.render_pixels(sc, views, pix, threads=cores)
    dt = time.perf_counter() - t
    offs = lf_inputs.pixel_offsets(views, pix)
    hit = idx[:, 0] >= 0
    psnr = {}
    for k, img in gpu_images.items():
        g = img.cpu().numpy().astype(np.float64)[offs]
        psnr[k] = oracle.psnr(ref, g, hit)
    psnr_k = {}
    if k_images:
        cont, chit = oracle.lobe_reference_pixels(cfg.lobes(), views, pix, threads=cores)
        cont[chit] += 0.005          # the mean of the texels' U(0, 0.01) noise
        for k, img in k_images.items():
            g = img.cpu().numpy().astype(np.float64)[offs]
            psnr_k[k] = oracle.psnr(cont, g, chit & hit)
    # whole frames of the two single-view cases: all cores, and one thread for the small one
    full = {}
    for c, single_too in ((lf_inputs.config_small(), True), (lf_inputs.config_precision(), False)):
        scf = oracle.Scene(c.M, c.N, c.C, "lobe", lobes=c.lobes())
        oracle.sf_points(c.M)
        oracle.sf_points(c.N)
        t_f = time.perf_counter()
        oracle.render_views(scf, c.views, threads=cores)
        entry = {"rays": c.rays, "table": f"{c.M:,} x {c.N:,}",
                 "all_cores_value": c.rays / (time.perf_counter() - t_f) / 1e9}
        if single_too:
            t_f = time.perf_counter()
            oracle.render_views(scf, c.views, threads=1)
            entry["single_thread_value"] = c.rays / (time.perf_counter() - t_f) / 1e9
        full[c.name] = entry
    # one host thread on a smaller sample (single-thread rate of the same oracle)
    pix1 = lf_inputs.sample_pixels(views, max(500, int(rate / cores * 2.0)), seed=13)
    t1 = time.perf_counter()
    oracle.render_pixels(sc, views, pix1, threads=1)
    single = len(pix1) / (time.perf_counter() - t1)
    base = {"value": n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": single / 1e9,
            "full_frames": full,
            "sample": f"{n:,} random pixels of orbit frame 0 ({hits:,} hits), brute-force FP64 K-NN "
                      f"over all {cfg.M:,}+{cfg.N:,} SF points, texels from the FP64 lobe field; "
                      f"{dt:.1f} s on {cores} threads; full_frames: every pixel of the small "
                      f"and precision cases' single views"}
    return base, psnr, psnr_k


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle as it stands, on the same workload
# ---------------------------------------------------------------------------
def run_reference(args, rank: int, world: int):
    import oracle
    cfg = lf_inputs.config_large()
    cores = host_cores()
    sc = oracle.Scene(cfg.M, cfg.N, 4, "lobe", lobes=cfg.lobes())
    oracle.sf_points(cfg.M)
    oracle.sf_points(cfg.N)
    per_step = max(500, int(args.ref_pixels))
    steps = []
    for k in range(args.warmup + args.steps):
        views = lf_inputs.orbit_frame(k % cfg.extra["frames"])
        pix = lf_inputs.sample_pixels(views, per_step, seed=100 + k)
        t = time.perf_counter()
        oracle.render_pixels(sc, views, pix, threads=cores)
        if k >= args.warmup:
            steps.append(time.perf_counter() - t)
    tot = sum(steps)
    value = per_step * len(steps) / tot / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(steps) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(cfg), "table_storage": "FP64 lobe field (oracle)",
                   "rays_per_step": per_step, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step:,} random pixels per step of the orbit frames"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="e4m3", choices=["e4m3", "f16", "f32"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-pixels", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick-tune", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--launch", default="", help="tile_w,tile_h,warp_w,order,persistent (skips the autotuner)")
    ap.add_argument("--workload", default="large",
                    choices=["large", "precision", "fit", "precompute", "post_filter"],
                    help="precision: 65,536 x 1,024 table, one 1920x1080 view (small profiling case); "
                         "fit: the differentiation leg alone (forward + backward + Adam per step); "
                         "precompute: the light-field precompute leg alone; "
                         "post_filter: the learned post-filter leg alone")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    if args.workload in ("fit", "precompute", "post_filter"):
        # the fit leg (data-parallel over the ranks), the precompute or the
        # post-filter leg alone (profiling cases of those kernels): one JSON object
        leg = {"fit": run_fit_steps, "precompute": run_precompute,
               "post_filter": run_post_filter}[args.workload](args)
        if rank == 0:
            print(json.dumps({args.workload: leg}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
