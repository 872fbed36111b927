"""Pins of the CPU oracle to facts outside itself (mathematics, the paper's printed
expressions, published reference values, library routines, brute force and
invariants). CPU only."""
import math
from fractions import Fraction
from math import isqrt

import numpy as np
import pytest

import lf_inputs
import oracle
from conftest import golden


def _golden_rows(name):
    rows = []
    with open(golden(name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                rows.append(ln.split())
    return rows


# --------------------------------------------------------------------------
# SF point set (Section 2, SF point set equation)
# --------------------------------------------------------------------------
def _exact_phase_53(i: int) -> float:
    """floor(2^53 * frac(i*(sqrt5-1)/2)) / 2^53 from exact integer arithmetic."""
    B = 400
    s5 = isqrt(5 << (2 * B))                 # floor(sqrt5 * 2^B)
    num = i * (s5 - (1 << B))                # i*(sqrt5-1)*2^B (within i)
    frac = num % (1 << (B + 1))              # frac of i*(sqrt5-1)/2, scaled by 2^(B+1)
    return (frac >> (B + 1 - 53)) / float(1 << 53)


def test_phase_is_golden_ratio_fraction():
    rng = np.random.default_rng(1)
    ids = [0, 1, 2, 3, 5, 8, 13, 987, 4095, 65535, 262143, (1 << 24) - 1]
    ids += [int(v) for v in rng.integers(0, 1 << 24, 300)]
    for i in ids:
        assert oracle.sf_phase(i) == _exact_phase_53(i), i
    assert abs(oracle.sf_phase(1) - 0.6180339887498948482) <= 2.0 ** -53


def test_golden_angle_between_consecutive_points():
    ga = float(_golden_rows("golden_angle.txt")[0][0])
    n = 4096
    P = oracle.sf_points(n)
    az = np.degrees(np.arctan2(P[:, 1], P[:, 0]))
    step = np.mod(az[1:] - az[:-1], 360.0)
    mid = slice(50, n - 51)
    np.testing.assert_allclose(step[mid], 360.0 - ga, atol=1e-9)


@pytest.mark.parametrize("n", [1, 2, 7, 256, 1000, 4096, 65536])
def test_sf_points_closed_form_invariants(n):
    P = oracle.sf_points(n)
    i = np.arange(n)
    # z_i = 1 - (2i+1)/n: n slabs of equal height (equal area, Archimedes)
    np.testing.assert_array_equal(P[:, 2], 1.0 - (2 * i + 1) / n)
    np.testing.assert_allclose(np.linalg.norm(P, axis=1), 1.0, atol=2e-16 * 8)
    # antipodal structure: z_{n-1-i} = -z_i (to rounding); phi_{n-1-i} + phi_i == phi_{n-1} mod 2pi
    np.testing.assert_allclose(P[::-1, 2], -P[:, 2], rtol=0, atol=4.5e-16)
    phi = np.arctan2(P[:, 1], P[:, 0])
    s = np.mod(phi[::-1] + phi - phi[-1] + math.pi, 2 * math.pi) - math.pi
    ok = np.hypot(P[:, 0], P[:, 1]) > 1e-6
    assert np.all(np.abs(s[ok & ok[::-1]]) < 1e-9)
    # p_0 lies in the x-z half plane (phi_0 = 0)
    assert P[0, 1] == 0.0 and P[0, 0] > 0.0


def test_point_count_above_height_is_area_fraction():
    n = 65536
    P = oracle.sf_points(n)
    for z0 in (-0.9, -0.3, 0.0, 0.5, 0.99):
        cnt = int(np.sum(P[:, 2] > z0))
        assert abs(cnt - n * (1 - z0) / 2) <= 1.0


# --------------------------------------------------------------------------
# Brute-force K-NN == library k-d tree
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 6, 9, 64, 257, 1024, 4096])
def test_knn_matches_kdtree(n):
    from scipy.spatial import cKDTree
    P = oracle.sf_points(n)
    tree = cKDTree(P)
    rng = np.random.default_rng(n)
    Q = rng.standard_normal((200, 3))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    for K in (1, 5, 9):
        for q in Q:
            idx, d2 = oracle.knn(P, q, K)
            dd, ii = tree.query(q, k=min(K, n))
            ii = np.atleast_1d(ii)
            dd = np.atleast_1d(dd)
            assert list(idx) == list(ii)
            np.testing.assert_allclose(np.sqrt(d2), dd, rtol=1e-12, atol=1e-15)


def test_knn_ties_go_to_smaller_index():
    P = np.array([[1.0, 0, 0], [0, 1.0, 0], [1.0, 0, 0], [0, 0, 1.0]])
    idx, d2 = oracle.knn(P, np.array([1.0, 0, 0]), 3)
    assert list(idx) == [0, 2, 1]


# --------------------------------------------------------------------------
# Camera ray and sphere intersection
# --------------------------------------------------------------------------
def test_camera_ray_geometry():
    W, H = 64, 48
    v = lf_inputs.look_at((0.3, -2.0, 1.1), (0.0, 0.1, 0.0), W, H)
    r, u, f = (np.array(a, np.float64) for a in (v.right, v.up, v.forward))
    ty = math.tan(math.radians(22.5))
    for (x, y) in [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (17, 30), (W // 2, H // 2)]:
        d = oracle.camera_ray(v, x, y).astype(np.float64)
        assert abs(np.linalg.norm(d) - 1) < 3e-7
        # pixel centres at +0.5; row 0 at the top (+up), column 0 on the left (-right)
        ex = (2 * (x + 0.5) / W - 1) * ty * W / H
        ey = (1 - 2 * (y + 0.5) / H) * ty
        assert abs(math.atan2(d @ r, d @ f) - math.atan(ex)) < 2e-6
        assert abs(math.atan2(d @ u, math.hypot(d @ f, d @ r)) -
                   math.atan2(ey, math.hypot(1, ex))) < 2e-6
    top = oracle.camera_ray(v, W // 2, 0).astype(np.float64)
    bot = oracle.camera_ray(v, W // 2, H - 1).astype(np.float64)
    assert top @ u > 0 > bot @ u
    left = oracle.camera_ray(v, 0, H // 2).astype(np.float64)
    assert left @ r < 0
    # full vertical angle between the centres of the first and last rows
    ang = math.acos(np.clip(top @ bot, -1, 1))
    nx, ny = ty * W / H / W, ty * (1 - 1 / H)
    want = math.acos((1 + nx * nx - ny * ny) / (1 + nx * nx + ny * ny))
    assert abs(ang - want) < 1e-5


def test_intersection_against_line_distance():
    rng = np.random.default_rng(7)
    R, O = 1.3, np.array([0.2, -0.4, 0.1])
    for _ in range(3000):
        e = O + rng.uniform(1.6, 4.0) * R * lf_inputs._random_dir(rng)
        d = rng.standard_normal(3)
        if rng.uniform() < 0.7:   # aim near the sphere
            d = (O + rng.uniform(-1.3, 1.3, 3) * R) - e
        d = (d / np.linalg.norm(d)).astype(np.float32)
        hit, ho, hd = oracle.intersect(R, O, e, d)
        ef, df = e.astype(np.float32).astype(np.float64), d.astype(np.float64)
        w = O - ef
        t_c = w @ df
        dist = np.linalg.norm(w - t_c * df)
        if abs(dist - R) < 1e-4 * R:
            continue
        assert hit == (dist < R and t_c > 0), (dist, R, t_c)
        if hit:
            for h in (ho, hd):
                assert abs(np.linalg.norm(h.astype(np.float64) - O) - R) < 2e-5 * R
            tn = (ho.astype(np.float64) - ef) @ df
            tf = (hd.astype(np.float64) - ef) @ df
            assert 0 < tn < tf
            half = math.sqrt(R * R - dist * dist)
            assert abs(tn - (t_c - half)) < 1e-4 and abs(tf - (t_c + half)) < 1e-4


def test_hit_fraction_matches_silhouette_cone():
    cfg = lf_inputs.config_small()
    v = cfg.views[0]
    f = np.array(v.forward, np.float64)
    half = math.asin(1.0 / 3.0)   # sphere radius R at distance 3R
    inside = clear = 0
    for y in range(0, v.height, 3):
        for x in range(0, v.width, 3):
            hit, d, *_ = oracle.trace_pixel(1.0, (0, 0, 0), v, x, y)
            a = math.acos(min(1.0, float(d.astype(np.float64) @ f)))
            if abs(a - half) < 1e-5:
                continue
            clear += 1
            assert hit == (a < half)
            inside += hit
    assert inside > 0.3 * clear


# --------------------------------------------------------------------------
# Filter kernel (Section 2)
# --------------------------------------------------------------------------
def test_kernel_size_equals_printed_expression():
    for R, N, size in _golden_rows("kernel_size.txt"):
        assert abs(float(R) * oracle.kernel_sigma(int(N)) - float(size)) < 1e-15 * float(size) * 4


def test_tent_weights_properties():
    n = 1024
    s = oracle.kernel_sigma(n)
    d = np.array([0.0, 0.3, 0.6, 0.99, 1.5]) * s
    w = oracle.tent_weights(d * d, n)
    raw = np.maximum(0, 1 - d / s)
    np.testing.assert_allclose(w, raw / raw.sum(), rtol=1e-14)
    assert w[-1] == 0.0 and abs(w.sum() - 1) < 1e-15
    # no point inside the kernel: the nearest takes all the weight
    w = oracle.tent_weights((np.array([1.1, 1.2, 1.3]) * s) ** 2, n)
    assert list(w) == [1.0, 0.0, 0.0]


# --------------------------------------------------------------------------
# Rendering (Section 2): constant table, linearity, separability, invariance
# --------------------------------------------------------------------------
def _tiny_views(W=40, H=32):
    return lf_inputs.pack_offsets([lf_inputs.look_at((2.2, 0.7, -0.4), (0, 0, 0), W, H),
                                   lf_inputs.look_at((-0.5, 1.9, 1.0), (0.05, 0, 0), 24, 20)])


def test_constant_table_renders_constant():
    M, N, Cc = 200, 60, 3
    views = _tiny_views()
    T = np.empty((M, N, Cc), np.float32)
    T[...] = np.array([0.25, 1.5, 3.0], np.float32)
    sc = oracle.Scene(M, N, Cc, "f32", T)
    out, idx, hits = oracle.render_views(sc, views)
    hit = idx[:, 0] >= 0
    assert hits == hit.sum() > 100
    np.testing.assert_allclose(out[hit], np.broadcast_to([0.25, 1.5, 3.0], out[hit].shape),
                               rtol=1e-14)
    assert np.all(out[~hit] == 0) and np.all(idx[~hit] == -1)


def test_render_linear_and_separable():
    M, N = 150, 40
    views = _tiny_views()
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, M)
    g = rng.uniform(0, 1, N)
    T = (f[:, None] * g[None, :]).astype(np.float32)[:, :, None]
    sc = oracle.Scene(M, N, 1, "f32", T)
    out, idx, _ = oracle.render_views(sc, views)
    # separable table: out = (sum_a Wo_a f(i_a)) * (sum_b Wd_b g(j_b))
    pix = lf_inputs.pixel_list(views)
    Po, Pd = oracle.sf_points(M), oracle.sf_points(N)
    checked = 0
    for p in pix[::7]:
        hit, _, _, _, qo, qd = oracle.trace_pixel(1.0, (0, 0, 0), views[p[0]], p[1], p[2])
        off = lf_inputs.pixel_offsets(views, p[None])[0]
        if not hit:
            assert out[off, 0] == 0
            continue
        io, d2o = oracle.knn(Po, qo, 5)
        jd, d2d = oracle.knn(Pd, qd, 5)
        wo, wd = oracle.tent_weights(d2o, M), oracle.tent_weights(d2d, N)
        want = float(wo @ f[io]) * float(wd @ g[jd])
        assert abs(out[off, 0] - want) < 2e-7 * abs(want)
        assert list(idx[off]) == list(io) + list(jd)
        checked += 1
    assert checked > 20
    # linearity in the table
    T2 = rng.uniform(-1, 1, (M, N, 1)).astype(np.float32)
    o2, _, _ = oracle.render_views(oracle.Scene(M, N, 1, "f32", T2), views)
    o3, _, _ = oracle.render_views(
        oracle.Scene(M, N, 1, "f32", (2 * T.astype(np.float64) - 3 * T2).astype(np.float32)), views)
    np.testing.assert_allclose(o3, 2 * out - 3 * o2, atol=1e-6)


def test_render_invariant_to_sphere_scale_and_translation():
    M, N = 300, 80
    rng = np.random.default_rng(5)
    T = rng.uniform(0, 1, (M, N, 3)).astype(np.float32)
    v = lf_inputs.look_at((2.0, -1.0, 0.5), (0, 0, 0), 48, 40)
    R, O = 2.0, np.array([1.0, -2.0, 0.5])
    v2 = lf_inputs.look_at(O + 2.0 * np.array([2.0, -1.0, 0.5]), O, 48, 40)
    a, ia, _ = oracle.render_views(oracle.Scene(M, N, 3, "f32", T), [v])
    b, ib, _ = oracle.render_views(oracle.Scene(M, N, 3, "f32", T, R=R, O=O), [v2])
    same = np.all(ia == ib, axis=1)
    assert same.mean() > 0.97
    np.testing.assert_allclose(a[same], b[same], atol=2e-4)


# --------------------------------------------------------------------------
# Backward: adjoint identity
# --------------------------------------------------------------------------
def test_backward_is_adjoint_of_render():
    M, N, Cc = 120, 50, 3
    views = _tiny_views(30, 24)
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, (M, N, Cc)).astype(np.float32)
    sc = oracle.Scene(M, N, Cc, "f32", x)
    pix = lf_inputs.pixel_list(views)
    Ax, _, hits = oracle.render_pixels(sc, views, pix)
    g = rng.standard_normal(Ax.shape)
    G = oracle.render_backward(sc, views, pix, g)
    lhs = float(np.sum(Ax * g))
    rhs = float(np.sum(x.astype(np.float64) * G))
    assert hits > 50
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    # each hit pixel distributes total weight 1 over its 25 texels
    G1 = oracle.render_backward(sc, views, pix, np.ones_like(g))
    assert abs(G1[..., 0].sum() - hits) < 1e-9 * hits


# --------------------------------------------------------------------------
# Quantisers against library conversions
# --------------------------------------------------------------------------
def test_f16_matches_numpy():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    dec = oracle.f16_decode(codes)
    ref = codes.view(np.float16).astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(dec))
    np.testing.assert_array_equal(dec[~nan], ref[~nan])
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-1, 1, 20000), rng.uniform(-1e-4, 1e-4, 5000),
                        rng.uniform(-7e-8, 7e-8, 2000)]).astype(np.float32)
    # midpoints between neighbouring binary16 values (ties to even)
    fin = ref[~nan & (np.abs(ref) <= 1.0)]
    fin = np.unique(fin)
    mids = ((fin[1:] + fin[:-1]) / 2).astype(np.float32)
    x = np.concatenate([x, mids[::7], fin.astype(np.float32)])
    np.testing.assert_array_equal(oracle.f16_encode(x), x.astype(np.float16).view(np.uint16))


def test_e4m3_matches_torch():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    dec = oracle.e4m3_decode(codes)
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(dec)) and nan.sum() == 2
    np.testing.assert_array_equal(dec[~nan], ref[~nan])
    fin = np.unique(ref[~nan])
    mids = ((fin[1:] + fin[:-1]) / 2)
    rng = np.random.default_rng(4)
    x = np.concatenate([fin, mids, rng.uniform(-448, 448, 20000), rng.uniform(-0.02, 0.02, 5000),
                        np.nextafter(mids, 0), np.nextafter(mids, 1000)]).astype(np.float32)
    x = x[np.abs(x) <= 448]
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(oracle.e4m3_encode(x), want)
    # saturation beyond the largest finite value
    assert list(oracle.e4m3_encode(np.array([449.0, 1e6, -500.0], np.float32))) == [0x7e, 0x7e, 0xfe]


@pytest.mark.parametrize("dtype", ["f16", "e4m3"])
def test_quantize_rows_scale_and_error(dtype):
    rng = np.random.default_rng(6)
    T = rng.uniform(0, 2, (37, 19, 4)).astype(np.float32)
    T[5] = 0.0
    codes, s = oracle.quantize_rows(T, dtype)
    amax = np.abs(T).reshape(37, -1).max(1)
    div = np.float32(448.0) if dtype == "e4m3" else np.float32(1.0)
    want = np.where(amax == 0, np.float32(1), (amax / div).astype(np.float32))
    np.testing.assert_array_equal(s, want)
    dec = (oracle.e4m3_decode if dtype == "e4m3" else oracle.f16_decode)(codes).reshape(T.shape)
    rel = 2.0 ** (-4 if dtype == "e4m3" else -11)
    err = np.abs(dec * s[:, None, None] - T)
    assert np.all(err <= rel * np.abs(T) + s[:, None, None] * (2.0 ** (-10 if dtype == "e4m3" else -25)))
    top = dec.reshape(37, -1).max(1)
    assert np.all(top[amax > 0] == (448.0 if dtype == "e4m3" else 1.0))


# --------------------------------------------------------------------------
# Lobe field input and its counter-based noise
# --------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    for seed, k, val in _golden_rows("splitmix64.txt"):
        assert oracle.splitmix64(int(seed), int(k)) == int(val)


def test_lobe_field_peak_and_noise():
    M, N = 64, 32
    P, Q = oracle.sf_points(M), oracle.sf_points(N)
    i, j = 10, 7
    d = Q[j] - P[i]
    d /= np.linalg.norm(d)
    lob = lf_inputs.Lobes(9, 1, 3, P[i][None].copy(), d[None].copy(), np.array([7.0]),
                          np.array([13.0]), np.array([[0.2, 0.5, 0.9]]), noise_seed=9)
    v = oracle.lobe_texel(lob, M, N, i, j)
    u = np.array([oracle.splitmix64(9, (i << 32) | (j << 4) | c) >> 11 for c in range(3)]) / 2.0**53
    np.testing.assert_allclose(v, [0.2, 0.5, 0.9] + 0.01 * u, rtol=1e-14)
    # with no lobes the table is 0.01 * U[0,1): mean 0.005, variance 1e-4/12
    none = lf_inputs.Lobes(3, 0, 4, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0),
                           np.zeros((0, 4)), noise_seed=3)
    T = oracle.lobe_table(none, 256, 64).astype(np.float64).ravel()
    assert T.min() >= 0 and T.max() < 0.01
    assert abs(T.mean() - 0.005) < 5e-5 and abs(T.var() - 1e-4 / 12) < 2e-7


def test_lobe_table_range():
    cfg = lf_inputs.config_small()
    lob = cfg.lobes()
    T = oracle.lobe_table(lob, cfg.M, cfg.N)
    assert T.min() >= 0
    assert np.all(T.max(axis=(0, 1)) <= lob.col.sum(0) + 0.01)


def test_psnr_definition():
    ref = np.array([[1.0, 0.5], [0.25, 0.0], [9.0, 9.0]])
    hit = np.array([True, True, False])
    assert oracle.psnr(ref, ref, hit) == float("inf")
    assert abs(oracle.psnr(ref, ref + 0.01, hit) - 10 * math.log10(1.0 / 1e-4)) < 1e-9


# --------------------------------------------------------------------------
# Upper-hemisphere storage (Section 3: only origins with z > 0 are stored)
# --------------------------------------------------------------------------
def test_upper_hemisphere_mode():
    M, N = 400, 90
    rng = np.random.default_rng(12)
    T = rng.uniform(0, 1, (M, N, 3)).astype(np.float32)
    top = lf_inputs.look_at((0.05, 0.1, 2.5), (0, 0, 0), 40, 40)
    bottom = lf_inputs.look_at((0.05, 0.1, -2.5), (0, 0, 0), 40, 40)
    full = oracle.Scene(M, N, 3, "f32", T)
    up = oracle.Scene(M, N, 3, "f32", T[:M // 2], upper=True)
    # seen from far above, every origin neighbour is stored: same image as the full table
    a, ia, ha = oracle.render_views(full, [top])
    b, ib, hb = oracle.render_views(up, [top])
    assert ha == hb > 500
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_allclose(a, b, atol=1e-12)
    # seen from below, every pixel is masked
    c, ic, hc = oracle.render_views(up, [bottom])
    assert hc == 0 and np.all(c == 0) and np.all(ic == -1)
    # an oblique view: a pixel is masked exactly when all 5 origin neighbours lie in the
    # lower half; a constant table renders its constant on every unmasked pixel
    side = lf_inputs.look_at((2.4, 0.3, 0.4), (0, 0, 0), 48, 48)
    K = np.full((M // 2, N, 3), 0.75, np.float32)
    o, io, h = oracle.render_views(oracle.Scene(M, N, 3, "f32", K, upper=True), [side])
    Po = oracle.sf_points(M)
    masked = partial = 0
    for p in lf_inputs.pixel_list([side])[::3]:
        hit, _, _, _, qo, _ = oracle.trace_pixel(1.0, (0, 0, 0), side, p[1], p[2])
        off = p[2] * 48 + p[1]
        if not hit:
            continue
        nn, _ = oracle.knn(Po, qo, 5)
        kept = nn < M // 2
        if not kept.any():
            masked += 1
            assert io[off, 0] == -1 and np.all(o[off] == 0)
        else:
            partial += int(not kept.all())
            assert list(io[off, :5]) == list(nn)
            np.testing.assert_allclose(o[off], 0.75, rtol=1e-12)
    assert masked > 10 and partial > 5
    w = oracle.tent_weights_kept(np.array([0.0, 0.01, 0.02, 0.03, 0.04]) ** 2,
                                 np.array([300, 10, 250, 20, 30]), M, M // 2)
    assert w[0] == 0 and w[2] == 0 and abs(w.sum() - 1) < 1e-15


# --------------------------------------------------------------------------
# Continuous lobe field (the reference of interpolation quality per K)
# --------------------------------------------------------------------------
def test_continuous_lobe_field_samples_to_the_table():
    # at the SF points and the chord direction the field plus the texel's noise is the texel
    lob = lf_inputs.draw_lobes(4, 6, 4)
    M, N = 300, 70
    Po, Pd = oracle.sf_points(M), oracle.sf_points(N)
    for i, j in [(0, 0), (17, 3), (299, 69), (150, 35)]:
        d = Pd[j] - Po[i]
        d /= np.linalg.norm(d)
        cont = oracle.lobe_continuous(lob, Po[i], d)
        noise = np.array([0.01 * (oracle.splitmix64(lob.noise_seed, (i << 32) | (j << 4) | c) >> 11) * 2.0 ** -53
                          for c in range(4)])
        np.testing.assert_allclose(cont + noise, oracle.lobe_texel(lob, M, N, i, j), rtol=0, atol=1e-15)


def test_continuous_lobe_field_peak_and_antipode():
    lob = lf_inputs.draw_lobes(8, 1, 3)
    a, b = lob.ap[0], lob.ad[0]
    # a . a = 1 to rounding, so the peak is exact to a few ulp of kp + kd
    np.testing.assert_allclose(oracle.lobe_continuous(lob, a, b), lob.col[0], rtol=1e-14, atol=0)
    want = lob.col[0] * math.exp(-2 * lob.kp[0]) * math.exp(-2 * lob.kd[0])
    np.testing.assert_allclose(oracle.lobe_continuous(lob, -a, -b), want, rtol=1e-13, atol=0)


def test_reference_pixels_follow_the_ray():
    lob = lf_inputs.draw_lobes(2, 5, 3)
    v = lf_inputs.look_at((2.5, 0.4, -0.3), (0, 0, 0), 40, 30)
    pix = lf_inputs.pixel_list([v])
    out, hit = oracle.lobe_reference_pixels(lob, [v], pix)
    assert 0 < hit.sum() < len(pix)
    for k in np.nonzero(hit)[0][::97]:
        _, _, _, _, qo, qd = oracle.trace_pixel(1.0, (0, 0, 0), v, pix[k, 1], pix[k, 2])
        u = (qd - qo) / np.linalg.norm(qd - qo)
        np.testing.assert_allclose(out[k], oracle.lobe_continuous(lob, qo, u), rtol=0, atol=1e-15)
    assert np.all(out[~hit] == 0)
