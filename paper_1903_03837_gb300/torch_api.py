"""Tensor-level API over the C ABI: PyTorch supplies device memory and the
current CUDA stream; the kernels of liblumipath.so do all of the work.

* ``LightField``: a table on the GPU (create / render, FP32 or binary16 image /
  backward, searching again or from the forward's indices / launch shape)
* ``RenderFunction``: ``torch.autograd.Function`` whose backward is the
  library's scatter-add kernel, fed with the forward's indices (for fitting a
  table to target views); ``fit_step``: one data-parallel fitting step
* ``precompute_table``: the light-field precompute of Section 2 (rays r_k with
  jittered origins through an analytic volume), on the GPU; ``render_volume``:
  the direct render of that volume along each pixel's ray (ground truth)
* ``fill_lobe_table``: the synthetic lobe radiance field, filled on the GPU
* ``quantize_table``: per-row FP16 / E4M3 storage of an FP32 table
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import torch

from . import lumipath as lp


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _need_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def total_pixels(views: Sequence) -> int:
    return max(int(v.out_offset) + int(v.width) * int(v.height) for v in views)


class LightField:
    """Light-field table L^(i,j) on the current CUDA device (Section 2).

    radiance: [M,N,C] float32, or FP16/E4M3 codes ([M,N,C] int16/uint8) with
    ``scales`` [M] float32. With ``borrow=True`` the library reads the tensor in
    place (it must stay alive; its contents may change between renders).
    """

    def __init__(self, radiance: torch.Tensor, dtype: str = "f32", scales: Optional[torch.Tensor] = None,
                 R: float = 1.0, O=(0.0, 0.0, 0.0), borrow: bool = False, n_origins: Optional[int] = None,
                 upper: bool = False, k_nearest: int = 5):
        _need_cuda(radiance, "radiance")
        if radiance.dim() != 3:
            raise ValueError("radiance must be [M, N, C]")
        rows, N, Cc = (int(s) for s in radiance.shape)
        M = int(n_origins) if n_origins is not None else (2 * rows if upper else rows)
        if (M // 2 if upper else M) != rows:
            raise ValueError(f"radiance has {rows} rows; expected {M // 2 if upper else M} for M={M}")
        ok = {"f32": (torch.float32,), "f16": (torch.int16, torch.float16),
              "e4m3": (torch.uint8, torch.int8, torch.float8_e4m3fn)}[dtype]
        if radiance.dtype not in ok:
            raise ValueError(f"radiance dtype {radiance.dtype} does not match storage {dtype}")
        if scales is not None:
            _need_cuda(scales, "scales")
        desc = lp.lf_table_desc()
        desc.radius = float(R)
        desc.center[:] = [float(o) for o in O]
        desc.n_origins, desc.n_directions, desc.channels = M, N, Cc
        desc.dtype = lp.DTYPES[dtype]
        desc.flags = (lp.LF_TABLE_BORROW if borrow else 0) | (lp.LF_TABLE_UPPER_HEMISPHERE if upper else 0)
        desc.k_nearest = int(k_nearest)
        self.K = int(k_nearest) or 5
        self.M, self.N, self.C, self.dtype, self.R, self.O = M, N, Cc, dtype, float(R), tuple(O)
        self.rows, self.upper = rows, bool(upper)
        self._keep = (radiance, scales) if borrow else None
        self.handle = lp.lf_create_table(desc, radiance.data_ptr(),
                                         scales.data_ptr() if scales is not None else None, _stream())

    # -- launch shape --------------------------------------------------------
    def set_launch(self, tile_w=16, tile_h=16, warp_w=8, order=0, persistent=0, ctas_per_sm=0):
        cfg = lp.lf_launch(tile_w, tile_h, warp_w, order, persistent, ctas_per_sm)
        lp.lf_set_launch(self.handle, cfg)

    def get_launch(self) -> dict:
        return lp.lf_get_launch(self.handle).as_dict()

    # -- rendering -------------------------------------------------------------
    def render(self, views: Sequence, out: Optional[torch.Tensor] = None, with_idx: bool = False,
               idx: Optional[torch.Tensor] = None,
               half: bool = False) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
        """Render `views` into out [P, C] (float32, or float16 with half=True:
        the FP32 result rounded once, lf_render_f16)."""
        P = total_pixels(views)
        odt = torch.float16 if half else torch.float32
        if out is None:
            out = torch.empty((P, self.C), dtype=odt, device="cuda")
        _need_cuda(out, "out")
        if out.numel() < P * self.C or out.dtype != odt:
            raise ValueError(f"out must be {odt} with at least P*C elements")
        if with_idx and idx is None:
            idx = torch.empty((P, 2 * self.K), dtype=torch.int32, device="cuda")
        if idx is not None:
            _need_cuda(idx, "idx")
            if idx.numel() < P * 2 * self.K or idx.dtype != torch.int32:
                raise ValueError("idx must be int32 with at least P*2K elements")
        vv = lp.make_views(views)
        fn = lp.lf_render_f16 if half else lp.lf_render
        fn(self.handle, vv, len(views), out.data_ptr(), idx.data_ptr() if idx is not None else None, _stream())
        return out, idx

    def render_backward(self, views: Sequence, grad_out: torch.Tensor,
                        grad_table: Optional[torch.Tensor] = None,
                        idx: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Accumulate d(loss)/d(table) into grad_table. With `idx` (the int32
        [P, 2K] indices a render of the same views wrote), the backward reuses
        them instead of searching again (lf_render_backward_idx)."""
        _need_cuda(grad_out, "grad_out")
        if grad_out.dtype != torch.float32 or grad_out.numel() < total_pixels(views) * self.C:
            raise ValueError("grad_out must be float32 [P, C]")
        if grad_table is None:
            grad_table = torch.zeros((self.rows, self.N, self.C), dtype=torch.float32, device="cuda")
        _need_cuda(grad_table, "grad_table")
        if grad_table.dtype != torch.float32 or grad_table.numel() != self.rows * self.N * self.C:
            raise ValueError("grad_table must be float32 [rows, N, C]")
        vv = lp.make_views(views)
        if idx is not None:
            _need_cuda(idx, "idx")
            if idx.dtype != torch.int32 or not idx.is_contiguous() or idx.numel() < total_pixels(views) * 2 * self.K:
                raise ValueError("idx must be a contiguous int32 tensor of at least P * 2K elements")
            lp.lf_render_backward_idx(self.handle, vv, len(views), grad_out.data_ptr(), idx.data_ptr(),
                                      grad_table.data_ptr(), _stream())
        else:
            lp.lf_render_backward(self.handle, vv, len(views), grad_out.data_ptr(), grad_table.data_ptr(),
                                  _stream())
        return grad_table

    def sync_status(self):
        lp.lf_sync_status(self.handle, _stream())

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            lp.lf_destroy(h)
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RenderFunction(torch.autograd.Function):
    """image = render(table); d(loss)/d(table) by the library's backward kernel.

    ``table`` must be the FP32 tensor that ``lf`` borrows (``borrow=True``)."""

    @staticmethod
    def forward(ctx, table: torch.Tensor, lf: LightField, views):
        ctx.lf, ctx.views = lf, views
        out, idx = lf.render(views, with_idx=True)      # the backward reuses the indices
        ctx.idx = idx
        return out

    @staticmethod
    def backward(ctx, grad):
        g = ctx.lf.render_backward(ctx.views, grad.contiguous(), idx=ctx.idx)
        ctx.idx = None
        return g, None, None


def render(table: torch.Tensor, lf: LightField, views) -> torch.Tensor:
    return RenderFunction.apply(table, lf, views)


def fit_step(lf, table: torch.Tensor, opt, views, target: torch.Tensor, idx: torch.Tensor,
             global_values: int) -> torch.Tensor:
    """One data-parallel fitting step of an FP32 table against target images:
    render this rank's views (keeping their sample indices), the gradient of
    the mean squared error over all ranks' `global_values` image values, the
    backward scatter from those indices into table.grad, one all-reduce of the
    gradient table, the optimiser step. Returns this rank's sum of squared
    errors (a 0-d tensor, not synchronised)."""
    from . import replicas
    opt.zero_grad(set_to_none=False)
    img, _ = lf.render(views, idx=idx)
    diff = img - target
    lf.render_backward(views, (2.0 / global_values) * diff, table.grad, idx=idx)
    replicas.allreduce_sum_(table.grad)
    opt.step()
    return (diff * diff).sum()


def save_fit_state(path: str, table: torch.Tensor, opt, step: int) -> None:
    """Checkpoint of a table fit: the FP32 table, the optimiser state and the
    step, written to `path` atomically (a temporary file, then a rename)."""
    import os
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save({"table": table.detach().cpu(), "opt": opt.state_dict(), "step": int(step)}, tmp)
    os.replace(tmp, path)


def load_fit_state(path: str, table: torch.Tensor, opt) -> int:
    """Restore a checkpoint of save_fit_state into `table` (in place) and `opt`;
    returns the step to continue from."""
    ck = torch.load(path, map_location="cpu", weights_only=True)
    if tuple(ck["table"].shape) != tuple(table.shape):
        raise ValueError(f"checkpoint table {tuple(ck['table'].shape)} does not match {tuple(table.shape)}")
    with torch.no_grad():
        table.copy_(ck["table"].to(table.device))
    opt.load_state_dict(ck["opt"])
    return int(ck["step"])


def fill_lobe_table(lobes, M: int, N: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP32 [M,N,C] lobe radiance field on the GPU (parameters from lf_inputs.draw_lobes)."""
    if out is None:
        out = torch.empty((M, N, lobes.C), dtype=torch.float32, device="cuda")
    _need_cuda(out, "out")
    lp.lf_fill_lobe_table(M, N, lobes.C, lobes.L, lobes.ap, lobes.ad, lobes.kp, lobes.kd, lobes.col,
                          lobes.noise_seed, out.data_ptr(), _stream())
    return out


def _volume_desc(volume, M: int, N: int, C: int, rows: int):
    """lf_precompute_desc and lf_blob array of a volume scene (`volume` as
    lf_inputs.Volume: mu, width, dens, emit, bg0, bg1, spp, steps, jitter,
    seed, R, O)."""
    B = len(volume.width)
    if B > lp.LF_PRECOMPUTE_MAX_BLOBS:
        raise ValueError(f"at most {lp.LF_PRECOMPUTE_MAX_BLOBS} blobs")
    blobs = (lp.lf_blob * max(B, 1))()
    for b in range(B):
        blobs[b].center[:] = [float(x) for x in volume.mu[b]]
        blobs[b].width = float(volume.width[b])
        blobs[b].density = float(volume.dens[b])
        blobs[b].emit[:] = [float(x) for x in volume.emit[b]]
    d = lp.lf_precompute_desc()
    d.radius = float(volume.R)
    d.center[:] = [float(x) for x in volume.O]
    d.n_origins, d.n_directions, d.channels, d.rows = M, N, C, rows
    d.spp, d.steps, d.jitter, d.n_blobs = int(volume.spp), int(volume.steps), int(volume.jitter), B
    d.seed = int(volume.seed) & (2**64 - 1)
    d.bg0[:] = [float(x) for x in volume.bg0]
    d.bg1[:] = [float(x) for x in volume.bg1]
    return d, blobs


def precompute_table(volume, M: int, N: int, C: int = 4, rows: Optional[int] = None,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP32 [rows, N, C] light field of an emission-absorption volume scene
    (Section 2: rays r_k with jittered origins; `volume` as lf_inputs.Volume:
    mu, width, dens, emit, bg0, bg1, spp, steps, jitter, seed, R, O)."""
    rows = M if rows is None else int(rows)
    if out is None:
        out = torch.empty((rows, N, C), dtype=torch.float32, device="cuda")
    _need_cuda(out, "out")
    if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != rows * N * C:
        raise ValueError("out must be a contiguous float32 tensor of rows * N * C elements")
    d, blobs = _volume_desc(volume, M, N, C, rows)
    lp.lf_precompute_table(d, blobs, out.data_ptr(), _stream())
    return out


def render_volume(volume, views: Sequence, C: int = 4, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Direct render [P, C] float32 of a volume scene along each pixel's ray
    (front hit on S to the far intersection, `volume.steps` midpoint steps, one
    sample): the ground truth of a light-field render of its precomputed table.
    Misses are 0."""
    P = total_pixels(views)
    if out is None:
        out = torch.empty((P, C), dtype=torch.float32, device="cuda")
    _need_cuda(out, "out")
    if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() < P * C:
        raise ValueError("out must be a contiguous float32 tensor of at least P * C elements")
    d, blobs = _volume_desc(volume, 1, 1, C, 1)
    lp.lf_render_volume(d, blobs, lp.make_views(views), len(views), out.data_ptr(), _stream())
    return out


def quantize_table(T: torch.Tensor, dtype: str) -> Tuple[torch.Tensor, torch.Tensor]:
    """Per-row FP16 / E4M3 codes [M,N,4] (int16 holding binary16 bits, or uint8)
    and scales [M] of an FP32 [M,N,C] table."""
    _need_cuda(T, "T")
    M, N, Cc = (int(s) for s in T.shape)
    codes = torch.empty((M, N, 4), dtype=torch.int16 if dtype == "f16" else torch.uint8, device=T.device)
    scales = torch.empty((M,), dtype=torch.float32, device=T.device)
    lp.lf_quantize_table(T.data_ptr(), M, N, Cc, lp.DTYPES[dtype], codes.data_ptr(), scales.data_ptr(), _stream())
    return codes, scales
