"""GPU parity of the sampling path against the CPU oracle (called through the C ABI).

Bar: sample indices bit-exact; colours within 1e-5 absolute for FP32 tables
(and for FP16/E4M3 tables against the oracle reading the same codes); the
quantiser's codes and scales bit-exact; the lobe fill equal to the oracle's
FP64 evaluation rounded to FP32.
"""
import math

import numpy as np
import pytest

import lf_inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATOL = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03837_gb300 import torch_api
    return torch_api


def gpu_render(api, T, dtype, views, scales=None, launch=None, R=1.0, O=(0, 0, 0)):
    T = np.ascontiguousarray(T)
    if T.dtype == np.uint16:
        T = T.view(np.int16)
    t = torch.from_numpy(T).cuda()
    s = torch.from_numpy(np.ascontiguousarray(scales)).cuda() if scales is not None else None
    lf = api.LightField(t, dtype, s, R=R, O=O)
    if launch:
        lf.set_launch(**launch)
    out, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    torch.cuda.synchronize()
    res = out.cpu().numpy(), idx.cpu().numpy()
    lf.close()
    return res


def check_parity(got, want, hit_check=True):
    out, idx = got
    o_out, o_idx = want
    mism = np.any(idx != o_idx, axis=1)
    assert mism.sum() == 0, f"{mism.sum()} rays with different indices; first {np.nonzero(mism)[0][:5]}"
    err = np.abs(out.astype(np.float64) - o_out)
    assert err.max() <= ATOL, f"max abs error {err.max():.3g}"
    if hit_check:
        assert (idx[:, 0] >= 0).sum() > 0


# --------------------------------------------------------------------------
# Small configuration: 1,024 x 256 RGB FP32, one 256x256 view at 3R
# --------------------------------------------------------------------------
def test_small_config_full_frame(api):
    cfg = lf_inputs.config_small()
    T = oracle.lobe_table(cfg.lobes(), cfg.M, cfg.N)
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(cfg.M, cfg.N, cfg.C, "f32", T), cfg.views)
    got = gpu_render(api, T, "f32", cfg.views)
    check_parity(got, (want_out, want_idx))
    assert hits == int((got[1][:, 0] >= 0).sum())


def test_lobe_fill_matches_oracle(api):
    for (M, N, Cc, L, seed) in [(1024, 256, 3, 8, 0), (300, 77, 4, 16, 5)]:
        lob = lf_inputs.draw_lobes(seed, L, Cc)
        want = oracle.lobe_table(lob, M, N)
        got = api.fill_lobe_table(lob, M, N).cpu().numpy()
        diff = got != want
        # FP64 exp of CUDA and of the C library may differ in the last bit, so a
        # rounding to FP32 can land one ulp apart in rare cases.
        assert diff.mean() < 1e-5
        if diff.any():
            ulps = np.abs(got.view(np.int32)[diff].astype(np.int64) - want.view(np.int32)[diff])
            assert ulps.max() <= 1


@pytest.mark.parametrize("dtype", ["f16", "e4m3"])
@pytest.mark.parametrize("Cc", [3, 4])
def test_quantizer_matches_oracle(api, dtype, Cc):
    rng = np.random.default_rng(Cc)
    T = rng.uniform(0, 3, (97, 131, Cc)).astype(np.float32)
    T[3] = 0
    T[7, 5, 1] = 1e-30
    T[9] *= 1e-6
    want_codes, want_s = oracle.quantize_rows(T, dtype)
    codes, s = api.quantize_table(torch.from_numpy(T).cuda(), dtype)
    codes, s = codes.cpu().numpy(), s.cpu().numpy()
    np.testing.assert_array_equal(s, want_s)
    codes = codes.view(np.uint16) if dtype == "f16" else codes
    np.testing.assert_array_equal(codes[..., :Cc], want_codes)
    assert np.all(codes[..., Cc:] == 0)


@pytest.mark.parametrize("dtype", ["f16", "e4m3"])
def test_quantized_render_matches_oracle_on_same_codes(api, dtype):
    cfg = lf_inputs.config_small()
    lob = lf_inputs.draw_lobes(3, 8, 4)
    T = oracle.lobe_table(lob, cfg.M, cfg.N)
    codes, s = oracle.quantize_rows(T, dtype)
    want_out, want_idx, _ = oracle.render_views(
        oracle.Scene(cfg.M, cfg.N, 4, dtype, codes, s), cfg.views)
    got = gpu_render(api, codes.view(np.uint16 if dtype == "f16" else np.uint8), dtype, cfg.views, scales=s)
    check_parity(got, (want_out, want_idx))


# --------------------------------------------------------------------------
# Edge cases: tiny and ragged point sets, poles, odd image sizes, many views
# --------------------------------------------------------------------------
def _edge_views():
    vs = [
        lf_inputs.look_at((0.0, 0.0, 2.2), (0, 0, 0), 33, 17),        # straight down the +z pole
        lf_inputs.look_at((0.0, 0.0, -1.6), (0, 0, 0), 29, 31),       # from below, close
        lf_inputs.look_at((2.0, 1.0, 0.3), (0, 0, 0), 1, 1),
        lf_inputs.look_at((0.2, -3.5, 0.9), (0.1, 0, 0), 13, 7),
        lf_inputs.look_at((1.2, 1.2, 1.2), (0, 0, 0.3), 40, 24),
        lf_inputs.look_at((0.01, 0.0, 5.0), (0, 0, 0), 24, 24),
        lf_inputs.look_at((0.2, 0.1, 0.3), (1.0, 0.5, 0.0), 20, 20),     # eye inside the sphere
        lf_inputs.look_at((0.0, 0.0, 3.0), (1.0, 0.0, 0.0), 64, 48),     # silhouette across the image
    ]
    return lf_inputs.pack_offsets(vs)


@pytest.mark.parametrize("M,N", [(1, 1), (2, 3), (5, 4), (7, 64), (128, 129), (129, 200), (300, 1000),
                                 (2000, 130)])
def test_edge_point_counts_and_views(api, M, N):
    rng = np.random.default_rng(M * 7 + N)
    T = rng.uniform(-1, 2, (M, N, 4)).astype(np.float32)
    views = _edge_views()
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 4, "f32", T), views)
    got = gpu_render(api, T, "f32", views)
    check_parity(got, (want_out, want_idx))


def test_sphere_off_origin_and_scaled(api):
    M, N = 3000, 500
    R, O = 2.5, (0.7, -1.1, 0.4)
    rng = np.random.default_rng(17)
    T = rng.uniform(0, 1, (M, N, 3)).astype(np.float32)
    views = lf_inputs.pack_offsets([
        lf_inputs.look_at(np.array(O) + (6.0, 1.0, 2.0), O, 64, 48),
        lf_inputs.look_at(np.array(O) + (-1.0, 0.5, 5.5), O, 31, 29)])
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 3, "f32", T, R=R, O=O), views)
    got = gpu_render(api, T, "f32", views, R=R, O=O)
    check_parity(got, (want_out, want_idx))


def test_many_views_split_across_launches(api):
    rng = np.random.default_rng(5)
    M, N = 4096, 512
    T = rng.uniform(0, 1, (M, N, 4)).astype(np.float32)
    views = []
    for _ in range(70):
        w, h = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        views.append(lf_inputs.look_at(rng.uniform(1.4, 4) * lf_inputs._random_dir(rng), (0, 0, 0), w, h))
    views = lf_inputs.pack_offsets(views)
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 4, "f32", T), views)
    got = gpu_render(api, T, "f32", views)
    check_parity(got, (want_out, want_idx))


LAUNCHES = [
    dict(tile_w=16, tile_h=16, warp_w=8),
    dict(tile_w=32, tile_h=8, warp_w=32),
    dict(tile_w=8, tile_h=32, warp_w=4),
    dict(tile_w=16, tile_h=4, warp_w=16),
    dict(tile_w=64, tile_h=4, warp_w=8, order=1),
    dict(tile_w=16, tile_h=16, warp_w=8, persistent=1),
    dict(tile_w=8, tile_h=8, warp_w=8, order=1, persistent=1, ctas_per_sm=3),
    dict(tile_w=32, tile_h=1, warp_w=32, persistent=1),
]


@pytest.mark.parametrize("launch", LAUNCHES)
def test_launch_shapes_give_identical_images(api, launch):
    rng = np.random.default_rng(9)
    M, N = 16384, 512
    T = rng.uniform(0, 1, (M, N, 4)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.0, -1.5, 0.7), (0, 0, 0), 123, 77),
                                    lf_inputs.look_at((0.3, 2.5, -1.0), (0, 0, 0), 65, 97),
                                    lf_inputs.look_at((0.0, 0.0, 2.0), (0, 0, 0), 40, 40)])
    base = gpu_render(api, T, "f32", views)
    got = gpu_render(api, T, "f32", views, launch=launch)
    np.testing.assert_array_equal(got[1], base[1])
    np.testing.assert_array_equal(got[0], base[0])
    # persistent launches re-arm their queue: a second render is identical
    again = gpu_render(api, T, "f32", views, launch=launch)
    np.testing.assert_array_equal(again[0], base[0])


# --------------------------------------------------------------------------
# Index step at large point counts: random rays against brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("M,N", [(65536, 1024), (262144, 4096), (1 << 22, 64), (4096, 1 << 18)])
def test_index_step_large_sets_sampled(api, M, N):
    views = lf_inputs.pack_offsets([lf_inputs.look_at((1.7, 0.6, -0.9), (0, 0, 0), 640, 480),
                                    lf_inputs.look_at((0.05, 0.02, 2.4), (0, 0, 0), 320, 320)])
    codes = torch.zeros((M, N, 4), dtype=torch.uint8, device="cuda")
    scales = torch.ones((M,), dtype=torch.float32, device="cuda")
    lf = api.LightField(codes, "e4m3", scales, borrow=True)
    _, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    idx = idx.cpu().numpy()
    lf.close()
    del codes
    torch.cuda.empty_cache()
    pix = lf_inputs.sample_pixels(views, 3000, seed=M)
    offs = lf_inputs.pixel_offsets(views, pix)
    sc = oracle.Scene(M, N, 4, "lobe", lobes=lf_inputs.draw_lobes(0, 0, 4))
    _, want_idx, hits = oracle.render_pixels(sc, views, pix)
    mism = np.any(idx[offs] != want_idx, axis=1)
    assert hits > 500
    assert mism.sum() == 0, f"{mism.sum()} of {len(pix)} rays differ"


@pytest.mark.parametrize("M,N", [(1 << 24, 4), (3, 1 << 24)])
def test_index_step_maximum_point_counts(api, M, N):
    """The largest sets the boundary accepts (2^24 points): FP32 lattice
    coordinates of a 16.7 M-point set against brute force on sampled rays."""
    views = lf_inputs.pack_offsets([lf_inputs.look_at((1.7, 0.6, -0.9), (0, 0, 0), 320, 240),
                                    lf_inputs.look_at((0.03, 0.01, 2.4), (0, 0, 0), 64, 64),
                                    lf_inputs.look_at((0.02, -0.04, -2.1), (0, 0, 0), 64, 64)])
    codes = torch.zeros((M, N, 4), dtype=torch.uint8, device="cuda")
    scales = torch.ones((M,), dtype=torch.float32, device="cuda")
    lf = api.LightField(codes, "e4m3", scales, borrow=True)
    _, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    idx = idx.cpu().numpy()
    lf.close()
    del codes
    torch.cuda.empty_cache()
    pix = lf_inputs.sample_pixels(views, 500, seed=M + N)
    offs = lf_inputs.pixel_offsets(views, pix)
    sc = oracle.Scene(M, N, 4, "lobe", lobes=lf_inputs.draw_lobes(0, 0, 4))
    _, want_idx, hits = oracle.render_pixels(sc, views, pix)
    mism = np.any(idx[offs] != want_idx, axis=1)
    assert hits > 100
    assert mism.sum() == 0, f"{mism.sum()} of {len(pix)} rays differ"


# --------------------------------------------------------------------------
# Backward: oracle gradient, adjoint identity, finite differences
# --------------------------------------------------------------------------
@pytest.mark.parametrize("Cc", [3, 4])
def test_backward_matches_oracle_gradient(api, Cc):
    M, N = 700, 150
    rng = np.random.default_rng(Cc + 40)
    T = rng.uniform(0, 1, (M, N, Cc)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.0, 0.4, 0.2), (0, 0, 0), 48, 40),
                                    lf_inputs.look_at((-0.4, 1.8, 1.1), (0, 0, 0), 37, 41)])
    P = lf_inputs.total_pixels(views)
    g = rng.standard_normal((P, Cc)).astype(np.float32)
    sc = oracle.Scene(M, N, Cc, "f32", T)
    pix = lf_inputs.pixel_list(views)
    offs = lf_inputs.pixel_offsets(views, pix)
    want = oracle.render_backward(sc, views, pix, g[offs].astype(np.float64))
    lf = api.LightField(torch.from_numpy(T).cuda(), "f32")
    G = lf.render_backward(views, torch.from_numpy(g).cuda()).cpu().numpy().astype(np.float64)
    lf.close()
    scale = np.abs(want).max()
    assert np.abs(G - want).max() <= 2e-6 * max(1.0, scale) * 10


def test_backward_adjoint_and_finite_differences(api):
    # finite-difference check on a 256 x 64 RGB table
    M, N, Cc = 256, 64, 3
    rng = np.random.default_rng(77)
    T = torch.from_numpy(rng.uniform(0, 1, (M, N, Cc)).astype(np.float32)).cuda()
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.2, 0.3, 0.5), (0, 0, 0), 64, 64),
                                    lf_inputs.look_at((0.2, -2.0, -0.8), (0, 0, 0), 48, 48)])
    P = lf_inputs.total_pixels(views)
    wts = torch.from_numpy(rng.standard_normal((P, Cc)).astype(np.float32)).cuda()
    lf = api.LightField(T, "f32", borrow=True)

    def loss():
        out, _ = lf.render(views)
        return float((out.double() * wts.double()).sum())

    G = lf.render_backward(views, wts).double()
    # adjoint identity <A x, g> = <x, A^T g>
    assert abs(loss() - float((T.double() * G).sum())) <= 1e-5 * abs(loss())
    nz = torch.nonzero(G.abs() > 1e-3)
    pick = nz[torch.randperm(len(nz), generator=torch.Generator().manual_seed(0))[:40].cuda()]
    h = 0.05
    for (i, j, c) in pick.tolist():
        old = float(T[i, j, c])
        T[i, j, c] = old + h
        lp = loss()
        T[i, j, c] = old - h
        lm = loss()
        T[i, j, c] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(G[i, j, c])) <= 1e-4 * max(1.0, abs(fd)), (i, j, c, fd, float(G[i, j, c]))
    lf.close()


def test_autograd_function_fits(api):
    from paper_1903_03837_gb300.torch_api import render
    M, N, Cc = 512, 128, 3
    lob = lf_inputs.draw_lobes(1, 6, Cc)
    gt = api.fill_lobe_table(lob, M, N)
    views = lf_inputs.pack_offsets([lf_inputs.look_at(2.5 * lf_inputs._random_dir(np.random.default_rng(k)),
                                                      (0, 0, 0), 64, 64) for k in range(6)])
    lf_gt = api.LightField(gt, "f32")
    target, _ = lf_gt.render(views)
    table = torch.zeros_like(gt, requires_grad=True)
    lf = api.LightField(table.detach(), "f32", borrow=True)
    opt = torch.optim.Adam([table], lr=2e-2)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        img = render(table, lf, views)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < 0.1 * losses[0]
    lf.close()
    lf_gt.close()


def test_status_word_clean_and_cpu_tensors_rejected(api):
    T = torch.rand((64, 32, 4), device="cuda")
    lf = api.LightField(T, "f32")
    lf.render([lf_inputs.look_at((2, 0, 0), (0, 0, 0), 16, 16)])
    lf.sync_status()
    with pytest.raises(ValueError):
        lf.render([lf_inputs.look_at((2, 0, 0), (0, 0, 0), 16, 16)], out=torch.zeros((256, 4)))
    lf.close()
    with pytest.raises(ValueError):
        api.LightField(torch.zeros((4, 4, 4)), "f32")


@pytest.mark.parametrize("M,N", [(1024, 256), (16384, 512), (262144, 4096)])
def test_index_step_stress_against_kdtree(api, M, N):
    """Millions of rays from random cameras: every index set equals the library
    k-d tree's 5 nearest (the oracle's brute force is pinned to it)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(M + 1)
    views = lf_inputs.pack_offsets([lf_inputs.look_at(rng.uniform(1.3, 4.0) * lf_inputs._random_dir(rng),
                                                      0.2 * rng.standard_normal(3), 640, 640)
                                    for _ in range(8)])
    codes = torch.zeros((M, N, 4), dtype=torch.uint8, device="cuda")
    lf = api.LightField(codes, "e4m3", torch.ones((M,), device="cuda"), borrow=True)
    _, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    idx = idx.cpu().numpy()
    lf.close()
    pix = lf_inputs.pixel_list(views)
    offs = lf_inputs.pixel_offsets(views, pix)
    idx = idx[offs]
    hit = idx[:, 0] >= 0
    qo = np.zeros((len(pix), 3))
    qd = np.zeros((len(pix), 3))
    # unit hit vectors from the oracle's FP32 ray / sphere step, for the hit rays
    sel = np.nonzero(hit)[0]
    sub = sel[:: max(1, len(sel) // 400000)]
    for k in sub:
        _, _, _, _, qo[k], qd[k] = oracle.trace_pixel(1.0, (0, 0, 0), views[pix[k, 0]], pix[k, 1], pix[k, 2])
    for P, q, cols in ((oracle.sf_points(M), qo, slice(0, 5)), (oracle.sf_points(N), qd, slice(5, 10))):
        _, nn = cKDTree(P).query(q[sub], k=5)
        bad = np.any(np.sort(idx[sub][:, cols], axis=1) != np.sort(nn, axis=1), axis=1)
        assert bad.sum() == 0, f"{bad.sum()} of {len(sub)} index sets differ from the k-d tree"
    assert len(sub) > 100000


@pytest.mark.parametrize("dtype", ["f32", "e4m3"])
def test_upper_hemisphere_table(api, dtype):
    M, N = 3001, 700
    rng = np.random.default_rng(31)
    T = rng.uniform(0, 1, (M // 2, N, 4)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 96, 80),
                                    lf_inputs.look_at((0.2, 0.1, 2.6), (0, 0, 0), 40, 40),
                                    lf_inputs.look_at((0.3, -0.2, -2.2), (0, 0, 0), 32, 32)])
    if dtype == "f32":
        sc = oracle.Scene(M, N, 4, "f32", T, upper=True)
        tab, scales = torch.from_numpy(T).cuda(), None
    else:
        codes, s = oracle.quantize_rows(T, "e4m3")
        sc = oracle.Scene(M, N, 4, "e4m3", codes, s, upper=True)
        tab, scales = torch.from_numpy(codes).cuda(), torch.from_numpy(s).cuda()
    want_out, want_idx, hits = oracle.render_views(sc, views)
    lf = api.LightField(tab, dtype, scales, n_origins=M, upper=True)
    out, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    check_parity((out.cpu().numpy(), idx.cpu().numpy()), (want_out, want_idx))
    # backward drops the unstored rows too
    g = torch.from_numpy(rng.standard_normal(out.shape).astype(np.float32)).cuda()
    G = lf.render_backward(views, g).cpu().numpy().astype(np.float64)
    pix = lf_inputs.pixel_list(views)
    offs = lf_inputs.pixel_offsets(views, pix)
    Gw = oracle.render_backward(oracle.Scene(M, N, 4, "f32", T, upper=True), views, pix,
                                g.cpu().numpy()[offs].astype(np.float64))
    assert np.abs(G - Gw).max() <= 2e-5 * max(1.0, np.abs(Gw).max())
    lf.close()


@pytest.mark.parametrize("M,N,upper", [(1024, 256, False), (65536, 1024, False), (3001, 700, True)])
def test_nearest_sampling_mode(api, M, N, upper):
    """k_nearest = 1: each hit takes its nearest SF point and the pixel the single
    texel L^(i, j) (Section 2, nearest sampling)."""
    rng = np.random.default_rng(M + N)
    rows = M // 2 if upper else M
    T = rng.uniform(0, 1, (rows, N, 4)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 96, 80),
                                    lf_inputs.look_at((0.2, 0.1, 2.6), (0, 0, 0), 40, 40)])
    want_out, want_idx, hits = oracle.render_views(oracle.Scene(M, N, 4, "f32", T, K=1, upper=upper), views)
    lf = api.LightField(torch.from_numpy(T).cuda(), "f32", n_origins=M, upper=upper, k_nearest=1)
    out, idx = lf.render(views, with_idx=True)
    lf.sync_status()
    got = (out.cpu().numpy(), idx.cpu().numpy())
    assert got[1].shape == (lf_inputs.total_pixels(views), 2)
    check_parity(got, (want_out, want_idx))
    lf.close()


# --------------------------------------------------------------------------
# Backward from the forward's indices (lf_render_backward_idx)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["rgba", "rgb", "upper", "nearest", "nine"])
def test_backward_from_indices_equals_search(api, case):
    M, N, Cc, upper, K = 1024, 256, 4, False, 5
    if case == "rgb":
        Cc = 3
    if case == "upper":
        M, upper = 3001, True
    if case == "nearest":
        K = 1
    if case == "nine":
        K = 9
    rows = M // 2 if upper else M
    rng = np.random.default_rng(len(case))
    T = rng.uniform(0, 1, (rows, N, Cc)).astype(np.float32)
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 96, 80),
                                    lf_inputs.look_at((0.1, 0.05, 2.6), (0, 0, 0), 48, 48)])
    lf = api.LightField(torch.from_numpy(T).cuda(), "f32", n_origins=M, upper=upper, k_nearest=K)
    P = lf_inputs.total_pixels(views)
    g = torch.from_numpy(rng.standard_normal((P, Cc)).astype(np.float32)).cuda()
    _, idx = lf.render(views, with_idx=True)
    G_idx = lf.render_backward(views, g, idx=idx).cpu().numpy().astype(np.float64)
    G_srch = lf.render_backward(views, g).cpu().numpy().astype(np.float64)
    lf.sync_status()
    # the same weights; only the order of the atomic additions differs
    assert np.abs(G_idx - G_srch).max() <= 1e-5 * max(1.0, np.abs(G_srch).max())
    pix = lf_inputs.pixel_list(views)
    offs = lf_inputs.pixel_offsets(views, pix)
    Gw = oracle.render_backward(oracle.Scene(M, N, Cc, "f32", T, K=K, upper=upper), views, pix,
                                g.cpu().numpy()[offs].astype(np.float64))
    assert np.abs(G_idx - Gw).max() <= 2e-5 * max(1.0, np.abs(Gw).max())
    assert np.abs(Gw).max() > 0
    lf.close()


def test_backward_from_indices_rejects_bad_indices(api):
    from paper_1903_03837_gb300 import lumipath as lp
    M, N = 512, 128
    T = torch.rand((M, N, 4), device="cuda")
    lf = api.LightField(T, "f32")
    views = [lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 32, 32)]
    _, idx = lf.render(views, with_idx=True)
    g = torch.ones((32 * 32, 4), device="cuda")
    bad = idx.clone()
    hit = torch.nonzero(bad[:, 0] >= 0)[0, 0]
    bad[hit, 1] = M + 7                       # out of range: skipped and reported, never read
    lf.render_backward(views, g, idx=bad)
    with pytest.raises(lp.LfError) as e:
        lf.sync_status()
    assert e.value.status == lp.LF_ERR_DEVICE_CHECK
    lf.sync_status()                          # the word was cleared
    with pytest.raises(ValueError):
        lf.render_backward(views, g, idx=idx[: 10])
    lf.close()


def test_misaligned_buffers_are_argument_errors(api):
    """Vector stores and loads need aligned buffers: a misaligned image, index or
    gradient buffer is rejected on the host (LF_ERR_INVALID_ARG), never launched."""
    from paper_1903_03837_gb300 import lumipath as lp
    T = torch.rand((256, 64, 4), device="cuda")
    lf = api.LightField(T, "f32")
    views = [lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 16, 16)]
    P = 256
    out_bad = torch.empty(P * 4 + 1, device="cuda")[1:]          # 4 bytes off a 16-byte boundary
    idx_bad = torch.empty(P * 10 + 1, dtype=torch.int32, device="cuda")[1:]
    g = torch.ones((P, 4), device="cuda")
    grad_bad = torch.zeros(256 * 64 * 4 + 1, device="cuda")[1:]
    with pytest.raises(lp.LfError) as e:
        lf.render(views, out=out_bad)
    assert e.value.status == lp.LF_ERR_INVALID_ARG
    with pytest.raises(lp.LfError) as e:
        lf.render(views, idx=idx_bad)
    assert e.value.status == lp.LF_ERR_INVALID_ARG
    with pytest.raises(lp.LfError) as e:
        lf.render_backward(views, g, grad_bad.view(256, 64, 4))
    assert e.value.status == lp.LF_ERR_INVALID_ARG
    lf.sync_status()                                              # nothing ran, nothing recorded
    out, _ = lf.render(views)                                     # aligned buffers still work
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    lf.close()


@pytest.mark.parametrize("dtype,Cc", [("e4m3", 4), ("f32", 3), ("f32", 4)])
def test_binary16_image_is_the_rounded_fp32_image(api, dtype, Cc):
    """lf_render_f16: the same render, each value rounded once to binary16 (RNE)."""
    M, N = 2048, 256
    rng = np.random.default_rng(Cc)
    T = rng.uniform(0, 2, (M, N, Cc)).astype(np.float32)
    if dtype == "e4m3":
        codes, scales = oracle.quantize_rows(T, "e4m3")
        lf = api.LightField(torch.from_numpy(codes).cuda(), "e4m3", torch.from_numpy(scales).cuda())
    else:
        lf = api.LightField(torch.from_numpy(T).cuda(), "f32")
    views = lf_inputs.pack_offsets([lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 96, 80),
                                    lf_inputs.look_at((0.1, 0.05, 2.6), (0, 0, 0), 33, 17)])
    out32, idx32 = lf.render(views, with_idx=True)
    out16, idx16 = lf.render(views, with_idx=True, half=True)
    lf.sync_status()
    assert out16.dtype == torch.float16
    assert torch.equal(idx16, idx32)
    assert torch.equal(out16, out32.half())          # torch's conversion rounds to nearest even
    assert (out16 != 0).any()
    lf.close()
