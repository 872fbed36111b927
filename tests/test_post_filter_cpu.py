"""The post-filter's training side on the CPU (PyTorch CPU tensors): its
forward equals the FP64 oracle's, its SSIM equals the benchmark's measure away
from the image border, and its training lowers the loss on a learnable task."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1903_03837_gb300 import post_filter as pf  # noqa: E402


def test_forward_equals_the_oracle():
    torch.manual_seed(0)
    w = pf.init_weights(3, device="cpu")
    W1, b1, W2, b2, W3, b3 = pf.unpack(w)
    W3.normal_(0, 0.1)
    b1.normal_(0, 0.05)
    f = torch.rand(1, 4, 19, 23)
    f[:, 3] = (torch.rand(19, 23) < 0.7).float()
    got = pf.forward_torch(w, f)[0].double().numpy()
    want = oracle.post_filter(w.numpy(), f[0].double().numpy())
    assert np.abs(got - want).max() < 1e-5


def test_ssim_map_agrees_with_the_benchmark_measure_inside():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (30, 34, 3))
    y = np.clip(x + rng.normal(0, 0.05, x.shape), 0, 1)
    m = pf.ssim_map(torch.from_numpy(x).permute(2, 0, 1)[None].float(),
                    torch.from_numpy(y).permute(2, 0, 1)[None].float())[0, 0].double().numpy()
    inner = np.zeros((30, 34), bool)
    inner[5:-5, 5:-5] = True                  # beyond the window's reach of the border padding
    assert abs(m[inner].mean() - bench.ssim_mean(x, y, inner, 1.0)) < 1e-5
    same = pf.ssim_map(torch.from_numpy(x).permute(2, 0, 1)[None].float(),
                       torch.from_numpy(x).permute(2, 0, 1)[None].float())
    assert torch.allclose(same, torch.ones_like(same), atol=1e-5)


def test_training_lowers_the_loss_on_a_learnable_task():
    # target = 0.8 x the input colour on hit pixels: within the filter's reach (W3 can
    # cancel a fifth of the colour through the ReLU layers of positive activations)
    g = torch.Generator().manual_seed(2)
    f = torch.rand(16, 4, 24, 24, generator=g)
    f[:, 3] = (torch.rand(16, 24, 24, generator=g) < 0.8).float()
    t = 0.8 * f[:, :3] * f[:, 3:4]
    w, hist = pf.train(f, t, steps=300, batch=8, lr=3e-3)
    assert hist[-1] < 0.3 * hist[0], hist
    assert w.numel() == pf.N_WEIGHTS
