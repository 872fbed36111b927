"""GPU parity of the learned post-filter (lf_post_filter, Section 2
post-processing) against the FP64 oracle, called through the C ABI.

The kernel runs all three layers on the tensor cores with FP16 operands (the
input colour, the two hidden layers' activations and the weights each rounded
once to FP16, relative error 2^-11) and FP32 accumulation; the residual adds
the FP32 input colour. The bar is the error that implies, per pixel and
channel, propagated through the layers from the oracle's own FP64
intermediates (`fp16_bound`): every FP16 rounding bounded by 2^-11 of its
value, the FP32 sums of at most 144 products by 2^-16 of the sum of their
magnitudes, ReLU 1-Lipschitz. The hit mask is the same FP32 ray/sphere test on
both sides (bit-exact, and exact in FP16).
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


U16 = 2.0 ** -11        # FP16 rounding
ACC = 2.0 ** -16        # FP32 accumulation of 144 products (144 * 2^-24 < 2^-16)


def fp16_bound(weights, feats):
    """Per-pixel bound [3, H, W] of |kernel - FP64 filter| for one view's features."""
    W1, b1, W2, b2, W3, b3 = oracle.post_unpack(weights)
    x = np.asarray(feats, np.float64)
    zero16, zero3 = np.zeros(16), np.zeros(3)
    e_x = U16 * np.abs(x)
    e_x[3] = 0.0                                                  # the hit mask is 0 or 1, exact
    ex1 = oracle.conv3x3(e_x, np.abs(W1), zero16)
    s1 = oracle.conv3x3(np.abs(x), np.abs(W1), zero16)
    h1 = np.maximum(oracle.conv3x3(x, W1, b1), 0.0)
    e1 = ex1 + (U16 + ACC) * (s1 + ex1)
    e_h1 = e1 + U16 * (h1 + e1)                                   # ReLU, then FP16
    s2 = oracle.conv3x3(h1, np.abs(W2), zero16)                   # sum of |w h1| per output
    h2 = np.maximum(oracle.conv3x3(h1, W2, b2), 0.0)
    e2 = oracle.conv3x3(e_h1, np.abs(W2), zero16) + (U16 + ACC) * (s2 + oracle.conv3x3(e_h1, np.abs(W2), zero16))
    e_h2 = e2 + U16 * (h2 + e2)                                   # ReLU, then FP16
    s3 = oracle.conv3x3(h2 + e_h2, np.abs(W3), zero3)
    e3 = oracle.conv3x3(e_h2, np.abs(W3), zero3) + (U16 + ACC) * s3
    out = oracle.post_filter(weights, x)
    return 1.05 * e3 + 1e-6 * (1.0 + np.abs(out))


@pytest.mark.parametrize("C", [4, 3])
def test_post_filter_matches_oracle(mods, C):
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, C)
    w = random_weights(pf, 1)
    out = pf.apply(w, views, img)
    torch.cuda.synchronize()
    got, src, wn = out.cpu().numpy(), img.cpu().numpy(), w.cpu().numpy()
    checked, worst = 0, 0.0
    for v in views:
        a, b = v.out_offset, v.out_offset + v.pixels
        feats = oracle.post_features(v, src[a:b])
        want = oracle.post_filter(wn, feats)
        tol = fp16_bound(wn, feats)
        g = got[a:b, :3].reshape(v.height, v.width, 3).transpose(2, 0, 1)
        err = np.abs(g - want)
        assert np.all(err <= tol), (v.width, v.height, float(err.max()), float((err / tol).max()))
        worst = max(worst, float(err.max()))
        if C == 4:
            np.testing.assert_array_equal(got[a:b, 3], src[a:b, 3])
        checked += int((want != 0).any(axis=0).sum())
    assert checked > 1000
    assert worst > 0.0                 # the FP16 operands do change the result


def _check_views(got, src, wn, views, C):
    """Every pixel of every view against the FP64 filter within the FP16 bound."""
    worst = 0.0
    for v in views:
        a, b = v.out_offset, v.out_offset + v.pixels
        feats = oracle.post_features(v, src[a:b])
        want = oracle.post_filter(wn, feats)
        tol = fp16_bound(wn, feats)
        g = got[a:b, :3].reshape(v.height, v.width, 3).transpose(2, 0, 1)
        err = np.abs(g - want)
        assert np.all(err <= tol), (v.width, v.height, float(err.max()), float((err / tol).max()))
        worst = max(worst, float(err.max()))
        if C == 4:
            np.testing.assert_array_equal(got[a:b, 3], src[a:b, 3])
    return worst


def test_post_filter_strips_and_chunks(mods):
    """Views wider than one 124-column strip and taller than one chunk: the
    strips' edges, the chunks' first rows (computed from the six rows before
    them) and the last, partial band of each view."""
    api, pf = mods
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.1, -1.0, 0.8), (0, 0, 0), 640, 481),
                                    lf_inputs.look_at((0.4, 2.3, -0.9), (0, 0, 0), 301, 250)])
    img = light_field_image(api, views, 4)
    w = random_weights(pf, 4)
    out = pf.apply(w, views, img)
    torch.cuda.synchronize()
    assert _check_views(out.cpu().numpy(), img.cpu().numpy(), w.cpu().numpy(), views, 4) > 0.0


def test_post_filter_unaligned_image_rows(mods):
    """An RGBA image 4-byte but not 16-byte aligned takes the scalar loads and
    stores: the same result as the aligned copy, bit for bit."""
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, 4)
    w = random_weights(pf, 5)
    P = img.shape[0]
    base = torch.zeros(P * 4 + 1, device="cuda")
    shifted = base[1:].view(P, 4)
    shifted.copy_(img)
    obase = torch.zeros(P * 4 + 1, device="cuda")
    oshift = obase[1:].view(P, 4)
    assert shifted.data_ptr() % 16 != 0 and oshift.data_ptr() % 16 != 0
    want = pf.apply(w, views, img)
    pf.apply(w, views, shifted, out=oshift)
    torch.cuda.synchronize()
    assert torch.equal(oshift, want)


def test_post_filter_full_frame_crops(mods):
    """A 1920 x 1080 frame (chunks of many steps, the launch the bench times):
    crops at the corners, the centre and across strip and chunk boundaries
    against the FP64 filter of the crop, on the crop's pixels whose 7 x 7
    neighbourhood lies inside the crop or beyond the frame's border."""
    api, pf = mods
    view = lf_inputs.look_at((2.2, -1.1, 0.9), (0, 0, 0), 1920, 1080)
    img = light_field_image(api, [view], 4)
    w = random_weights(pf, 6)
    out = pf.apply(w, [view], img).cpu().numpy()
    src = img.cpu().numpy()
    wn = w.cpu().numpy()
    W, H = view.width, view.height
    crops = [(0, 0), (W - 40, H - 40), (W // 2 - 20, H // 2 - 20), (124 * 7 - 20, 60 * 9 - 20), (0, H - 40),
             (124 * 15 - 20, 200)]
    for xa, ya in crops:
        x0, y0 = max(xa - 3, 0), max(ya - 3, 0)
        x1, y1 = min(xa + 43, W), min(ya + 43, H)
        feats = np.zeros((4, y1 - y0, x1 - x0))
        for y in range(y0, y1):
            row = src[y * W + x0:y * W + x1, :3]
            feats[:3, y - y0] = row.T
            for x in range(x0, x1):
                feats[3, y - y0, x - x0] = 1.0 if oracle.trace_pixel(1.0, (0.0, 0.0, 0.0), view, x, y)[0] else 0.0
        want = oracle.post_filter(wn, feats)
        tol = fp16_bound(wn, feats)
        g = np.stack([out[y * W + x0:y * W + x1, :3] for y in range(y0, y1)]).transpose(2, 0, 1)
        ix0, iy0 = (3 if x0 > 0 else 0), (3 if y0 > 0 else 0)
        ix1, iy1 = (x1 - x0) - (3 if x1 < W else 0), (y1 - y0) - (3 if y1 < H else 0)
        err = np.abs(g - want)[:, iy0:iy1, ix0:ix1]
        assert np.all(err <= tol[:, iy0:iy1, ix0:ix1]), (xa, ya, float(err.max()))
        np.testing.assert_array_equal(np.stack([out[y * W + x0:y * W + x1, 3] for y in range(y0, y1)]),
                                      np.stack([src[y * W + x0:y * W + x1, 3] for y in range(y0, y1)]))


def test_post_filter_matches_the_training_forward(mods):
    api, pf = mods
    views = views_mix()
    img = light_field_image(api, views, 4)
    w = random_weights(pf, 2)
    out = pf.apply(w, views, img)
    src = img.cpu().numpy()
    wn = w.cpu().numpy()
    for v in views:
        a, b = v.out_offset, v.out_offset + v.pixels
        feats = oracle.post_features(v, src[a:b])
        f = torch.from_numpy(feats).float().cuda()[None]
        with torch.backends.cudnn.flags(enabled=True, allow_tf32=False):   # FP32 products
            want = pf.forward_torch(w, f)[0]
        g = out[a:b, :3].reshape(v.height, v.width, 3).permute(2, 0, 1)
        # the training forward is FP32 throughout: within 2e-5 of the FP64 filter,
        # so the kernel is within the FP16 bound plus that of it
        tol = torch.from_numpy(fp16_bound(wn, feats)).float().cuda() + 2e-5 * (1.0 + want.abs())
        assert bool(((g - want).abs() <= tol).all()), float((g - want).abs().max())


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
