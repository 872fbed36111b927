"""GPU parity of the learned post-filter (lf_post_filter, Section 2
post-processing) against the FP64 oracle, called through the C ABI.

Bar: |GPU - oracle| <= 2e-5 (1 + |oracle|) per channel. The kernel sums each
layer in FP32 (36, 144 and 144 products per output): with activations and
weights of order 1 the accumulated rounding stays below 1e-5 of the output's
scale; the hit mask is the same FP32 ray/sphere test on both sides (bit-exact).
"""
import numpy as np
import pytest

import lf_inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03837_gb300 import post_filter, torch_api
    return torch_api, post_filter


def views_mix():
    return lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 37, 29),
                                   lf_inputs.look_at((0.2, 0.1, 2.6), (0, 0, 0), 16, 16),
                                   lf_inputs.look_at((0.3, 0.2, 0.1), (0, 0, 0), 20, 12),     # eye inside S
                                   lf_inputs.look_at((-3.0, 0.5, 0.2), (0, 0, 0), 70, 33)])


def random_weights(pf, seed):
    w = pf.init_weights(seed)
    W1, b1, W2, b2, W3, b3 = pf.unpack(w)
    g = torch.Generator(device="cpu").manual_seed(seed + 5)
    W3.copy_(torch.randn(W3.shape, generator=g) * 0.1)
    for b in (b1, b2, b3):
        b.copy_(torch.randn(b.shape, generator=g) * 0.05)
    return w


def light_field_image(api, views, C):
    lob = lf_inputs.draw_lobes(3, 8, 4)
    T = api.fill_lobe_table(lob, 1024, 256)
    lf = api.LightField(T, "f32", borrow=True)
    img, _ = lf.render(views)
    lf.sync_status()
    lf.close()
    return img[:, :C].contiguous()


@pytest.mark.parametrize("C", [4, 3])
def test_post_filter_matches_oracle(mods, C):
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, C)
    w = random_weights(pf, 1)
    out = pf.apply(w, views, img)
    torch.cuda.synchronize()
    got, src, wn = out.cpu().numpy(), img.cpu().numpy(), w.cpu().numpy()
    checked = 0
    for v in views:
        a, b = v.out_offset, v.out_offset + v.pixels
        want = oracle.post_filter(wn, oracle.post_features(v, src[a:b]))
        g = got[a:b, :3].reshape(v.height, v.width, 3).transpose(2, 0, 1)
        err = np.abs(g - want)
        assert np.all(err <= 2e-5 * (1.0 + np.abs(want))), (v.width, v.height, float(err.max()))
        if C == 4:
            np.testing.assert_array_equal(got[a:b, 3], src[a:b, 3])
        checked += int((want != 0).any(axis=0).sum())
    assert checked > 1000


def test_post_filter_matches_the_training_forward(mods):
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, 4)
    w = random_weights(pf, 2)
    out = pf.apply(w, views, img)
    src = img.cpu().numpy()
    for v in views:
        a, b = v.out_offset, v.out_offset + v.pixels
        f = torch.from_numpy(oracle.post_features(v, src[a:b])).float().cuda()[None]
        with torch.backends.cudnn.flags(enabled=True, allow_tf32=False):   # FP32 products, as the kernel
            want = pf.forward_torch(w, f)[0]
        g = out[a:b, :3].reshape(v.height, v.width, 3).permute(2, 0, 1)
        assert torch.allclose(g, want, rtol=2e-5, atol=2e-5), float((g - want).abs().max())


def test_zero_last_layer_passes_the_image_through(mods):
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, 4)
    w = random_weights(pf, 3)
    W1, b1, W2, b2, W3, b3 = pf.unpack(w)
    W3.zero_()
    b3.zero_()
    out = pf.apply(w, views, img).cpu().numpy()
    src = img.cpu().numpy()
    # the render stores 0 for misses and the filter keeps hit pixels' colour: the same image
    np.testing.assert_array_equal(out, src)


def test_training_lowers_the_loss(mods):
    api, pf = mods
    cfg = lf_inputs.config_post_filter(n_train=4, n_test=1)
    feats, targets, _ = pf.make_pairs(cfg.extra["train"], cfg.M, cfg.N)
    assert feats.shape == (32, 4, 128, 128) and targets.shape == (32, 3, 128, 128)
    w, hist = pf.train(feats, targets, steps=300, batch=8)
    assert hist[-1] < 0.8 * hist[0], hist
