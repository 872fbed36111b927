"""The image-quality measures of the benchmark (no GPU): the structural
similarity index against its definition (Wang, Bovik, Sheikh, Simoncelli,
IEEE TIP 2004) -- the measure the paper reports against its path-traced ground
truth (Section 3) -- the PSNR helper, and the byte counts behind the roofline
(algorithmic bytes per ray, compulsory 32-byte sectors of a frame)."""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")
import bench  # noqa: E402

SIGMA = 1.5


def brute_ssim_at(x, y, i, j, L):
    """SSIM at pixel (i, j) of single-channel images from the definition: local
    means, variances and covariance under the 11 x 11 Gaussian window of
    standard deviation 1.5 (weights normalised to sum 1), then the index."""
    r = np.arange(-5, 6)
    w = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2 * SIGMA ** 2))
    w /= w.sum()
    a = x[i - 5:i + 6, j - 5:j + 6]
    b = y[i - 5:i + 6, j - 5:j + 6]
    mx, my = (w * a).sum(), (w * b).sum()
    vx = (w * (a - mx) ** 2).sum()
    vy = (w * (b - my) ** 2).sum()
    cxy = (w * (a - mx) * (b - my)).sum()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    return ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx ** 2 + my ** 2 + c1) * (vx + vy + c2))


def test_ssim_of_an_image_with_itself_is_one():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (40, 50, 3))
    assert abs(bench.ssim_mean(x, x, np.ones((40, 50), bool), 1.0) - 1.0) < 1e-12


def test_ssim_of_two_constant_images_is_the_luminance_term():
    a, b, L = 0.3, 0.7, 1.0
    x = np.full((30, 30, 3), a)
    y = np.full((30, 30, 3), b)
    c1 = (0.01 * L) ** 2
    want = (2 * a * b + c1) / (a * a + b * b + c1)
    got = bench.ssim_mean(x, y, np.ones((30, 30), bool), L)
    assert abs(got - want) < 1e-9


def test_ssim_matches_the_windowed_definition_away_from_the_border():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (32, 32, 1))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    for i, j in [(10, 10), (16, 20), (21, 12)]:
        mask = np.zeros((32, 32), bool)
        mask[i, j] = True
        got = bench.ssim_mean(x, y, mask, 1.0)
        want = brute_ssim_at(x[:, :, 0], y[:, :, 0], i, j, 1.0)
        assert abs(got - want) < 1e-6, (i, j, got, want)


def test_ssim_averages_channels_and_only_the_masked_pixels():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (24, 24, 3))
    y = x.copy()
    y[:12, :, 1] = rng.uniform(0, 1, (12, 24))     # damage one channel in the top half
    top = np.zeros((24, 24), bool)
    top[3:8, :] = True
    bottom = np.zeros((24, 24), bool)
    bottom[17:22, :] = True
    assert abs(bench.ssim_mean(x, y, bottom, 1.0) - 1.0) < 1e-12
    s_top = bench.ssim_mean(x, y, top, 1.0)
    one = bench.ssim_mean(x[:, :, 1:2], y[:, :, 1:2], top, 1.0)
    assert abs(s_top - (2.0 + one) / 3.0) < 1e-12 and one < 0.5


def test_psnr_helper():
    ref = np.array([[1.0, 0.5], [0.25, 0.0]])
    test = ref + 0.1
    hit = np.array([True, False])
    assert abs(bench.psnr_db(ref, test, hit) - 10 * math.log10(1.0 / 0.01)) < 1e-9


def test_algorithmic_bytes_per_ray():
    # per hit ray: 25 texels + 5 row scales (quantised tables) + the 16-byte pixel; a miss: the pixel
    assert bench.algorithmic_bytes(1, 1, "e4m3") == 25 * 4 + 5 * 4 + 16 == 136
    assert bench.algorithmic_bytes(1, 1, "f16") == 25 * 8 + 5 * 4 + 16 == 236
    assert bench.algorithmic_bytes(1, 1, "f32") == 25 * 16 + 16 == 416
    assert bench.algorithmic_bytes(0, 10, "e4m3") == 160


def test_compulsory_bytes_counts_distinct_sectors():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    N, rays = 37, 50
    idx = rng.integers(0, 20, (12, 10)).astype(np.int32)
    idx[3, 2] = -1                       # a missing origin neighbour
    got = bench.compulsory_bytes(torch.from_numpy(idx), N, rays, "e4m3")
    tex, sca = set(), set()
    for r in idx:
        for a in r[:5]:
            if a < 0:
                continue
            sca.add((int(a) * 4) // 32)
            for b in r[5:]:
                if b >= 0:
                    tex.add(((int(a) * N + int(b)) * 4) // 32)
    assert got["texel_sectors"] == len(tex) and got["scale_sectors"] == len(sca)
    assert got["bytes"] == rays * 16 + 32 * (len(tex) + len(sca))
