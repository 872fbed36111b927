"""Learned post-filter of the light-field image (Section 2, post-processing: a
network that removes the interpolation artifacts of the rendered image).

Inference runs in the library (``lf_post_filter``, a hand-written CUDA kernel:
three 3x3 convolution layers, 4 -> 16 -> 16 -> 3 channels, ReLU after the
first two, the result added to the input colour of the pixels whose ray meets
S). This module holds the weights and their training:

* training pairs: the light-field render of a precomputed table of an analytic
  volume scene (the input) and the direct render of the same volume (the
  target), compared on the pixels whose ray meets S -- the pixels the light
  field covers, as the paper masks the uncovered ones;
* the loss: the paper's generator loss, the squared error plus (1 - SSIM), over
  those pixels; the adversarial part of the paper's training is not built;
* the optimiser: Adam.

The training forward is PyTorch's convolution (the same sums as the kernel's,
in another order); training is not on the render path.
"""
from __future__ import annotations

import ctypes
import math
from typing import List, Sequence, Tuple

import torch
import torch.nn.functional as F

from . import lumipath as lp
from . import torch_api as api

HIDDEN = 16
SHAPES = [("W1", (HIDDEN, 4, 3, 3)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN, 3, 3)), ("b2", (HIDDEN,)),
          ("W3", (3, HIDDEN, 3, 3)), ("b3", (3,))]
N_WEIGHTS = sum(math.prod(s) for _, s in SHAPES)
assert N_WEIGHTS == lp.LF_POST_WEIGHTS


def unpack(w: torch.Tensor):
    """Views of the flat weight vector as (W1, b1, W2, b2, W3, b3)."""
    out, k = [], 0
    for _, s in SHAPES:
        n = math.prod(s)
        out.append(w[k:k + n].view(s))
        k += n
    return out


def init_weights(seed: int = 0, device: str = "cuda") -> torch.Tensor:
    """He-initialised hidden layers; a last layer of small weights, so the
    untrained filter is close to the identity on hit pixels."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for name, s in SHAPES:
        if name.startswith("b"):
            parts.append(torch.zeros(s))
        else:
            std = math.sqrt(2.0 / (s[1] * 9)) if name != "W3" else 1e-3
            parts.append(torch.randn(s, generator=g) * std)
    return torch.cat([p.reshape(-1) for p in parts]).to(device=device, dtype=torch.float32).contiguous()


def forward_torch(w: torch.Tensor, feats: torch.Tensor) -> torch.Tensor:
    """The filter on feature images [B, 4, H, W] (R, G, B, hit): [B, 3, H, W],
    the input colour plus the network's output on hit pixels, 0 elsewhere."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    h = F.relu(F.conv2d(feats, W1, b1, padding=1))
    h = F.relu(F.conv2d(h, W2, b2, padding=1))
    r = F.conv2d(h, W3, b3, padding=1)
    return (feats[:, :3] + r) * feats[:, 3:4]


def _gauss_window(device) -> torch.Tensor:
    r = torch.arange(-5, 6, dtype=torch.float32, device=device)
    g = torch.exp(-(r * r) / (2 * 1.5 ** 2))
    g = g / g.sum()
    return (g[:, None] * g[None, :])[None, None]


def ssim_map(x: torch.Tensor, y: torch.Tensor, data_range: float = 1.0) -> torch.Tensor:
    """Per-pixel SSIM (Wang et al., 2004; Gaussian window of standard deviation
    1.5 over 11 x 11, zero padding) of [B, C, H, W] images, averaged over C."""
    C = x.shape[1]
    win = _gauss_window(x.device).expand(C, 1, 11, 11)
    g = lambda a: F.conv2d(a, win, padding=5, groups=C)
    mx, my = g(x), g(y)
    vx = g(x * x) - mx * mx
    vy = g(y * y) - my * my
    cxy = g(x * y) - mx * my
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    m = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    return m.mean(dim=1, keepdim=True)


def loss_fn(out: torch.Tensor, target: torch.Tensor, mask: torch.Tensor, ssim_weight: float = 0.01):
    """Squared error plus ssim_weight * (1 - SSIM), both over the hit pixels."""
    n = mask.sum().clamp_min(1.0)
    mse = (((out - target) ** 2) * mask).sum() / (3.0 * n)
    ssim = (ssim_map(out, target) * mask).sum() / n
    return mse + ssim_weight * (1.0 - ssim), mse, ssim


def view_images(views: Sequence, flat: torch.Tensor, C: int) -> List[torch.Tensor]:
    """Per-view [C, H, W] images of a flat [P, C] buffer."""
    out = []
    for v in views:
        a = flat[v.out_offset:v.out_offset + v.width * v.height, :C]
        out.append(a.reshape(v.height, v.width, C).permute(2, 0, 1))
    return out


def make_pairs(scenes, M: int, N: int) -> Tuple[torch.Tensor, torch.Tensor, list]:
    """(features [B, 4, H, W], targets [B, 3, H, W], per-scene (volume, views,
    flat light-field image)) of every view of `scenes` (a list of (volume,
    views), views of one size): the light-field render of each scene's
    precomputed M x N table, the hit mask from its index output, and the direct
    render of the volume."""
    feats, targets, flats = [], [], []
    for vol, views in scenes:
        T = api.precompute_table(vol, M, N, 4)
        lf = api.LightField(T, "f32", borrow=True)
        img, idx = lf.render(views, with_idx=True)
        lf.sync_status()
        lf.close()
        gt = api.render_volume(vol, views, 4)
        hit = (idx[:, :1] >= 0).float()
        for a, m, t in zip(view_images(views, img, 3), view_images(views, hit, 1), view_images(views, gt, 3)):
            feats.append(torch.cat([a, m], 0))
            targets.append(t)
        flats.append((vol, views, img))
        del T
    return torch.stack(feats), torch.stack(targets), flats


def train(feats: torch.Tensor, targets: torch.Tensor, steps: int = 2000, batch: int = 16, lr: float = 1e-3,
          seed: int = 0) -> Tuple[torch.Tensor, List[float]]:
    """Adam on random batches of the training views; returns the weights and
    the loss every 100 steps."""
    w = init_weights(seed, device=str(feats.device)).requires_grad_(True)
    opt = torch.optim.Adam([w], lr=lr)
    g = torch.Generator(device="cpu").manual_seed(seed + 1)
    history = []
    for step in range(steps):
        pick = torch.randint(0, feats.shape[0], (batch,), generator=g).to(feats.device)
        x, t = feats[pick], targets[pick]
        loss, _, _ = loss_fn(forward_torch(w, x), t, x[:, 3:4])
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        if step % 100 == 0 or step == steps - 1:
            history.append(float(loss.detach()))
    return w.detach().contiguous(), history


class PostFilter:
    """Trained weights ready for the library's post-filter (a host copy: the
    kernel takes them in its parameter block)."""

    def __init__(self, w: torch.Tensor):
        if w.numel() != N_WEIGHTS:
            raise ValueError(f"weights must have {N_WEIGHTS} values")
        flat = w.detach().to("cpu", torch.float32).reshape(-1).tolist()
        self.host = (ctypes.c_float * N_WEIGHTS)(*flat)

    def __call__(self, views: Sequence, image: torch.Tensor, R: float = 1.0, O=(0.0, 0.0, 0.0),
                 out: torch.Tensor = None) -> torch.Tensor:
        """The filter of a flat [P, C] light-field image of `views` (lf_post_filter)
        into a new [P, C] image."""
        api._need_cuda(image, "image")
        if image.dtype != torch.float32 or image.dim() != 2:
            raise ValueError("image must be a float32 [P, C] tensor")
        if out is None:
            out = torch.empty_like(image)
        api._need_cuda(out, "out")
        lp.lf_post_filter(R, O, int(image.shape[1]), self.host, lp.make_views(views), len(views),
                          image.data_ptr(), out.data_ptr(), api._stream())
        return out


def apply(w: torch.Tensor, views: Sequence, image: torch.Tensor, R: float = 1.0, O=(0.0, 0.0, 0.0),
          out: torch.Tensor = None) -> torch.Tensor:
    """One-off use of PostFilter(w)."""
    return PostFilter(w)(views, image, R, O, out)
