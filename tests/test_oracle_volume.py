"""Pins of the light-field precompute oracle (Section 2) against facts that do
not come from the oracle itself: closed forms of the emission-absorption
integral, the geometry of the ray r_k and of the jitter disk, invariances and
the convergence order of the midpoint rule."""
import math

import numpy as np
import pytest

import lf_inputs
import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def vol(mu, width, dens, emit, **kw):
    kw.setdefault("spp", 1)
    kw.setdefault("steps", 64)
    kw.setdefault("jitter", 0)
    return lf_inputs.Volume(np.asarray(mu, float).reshape(-1, 3), np.asarray(width, float),
                            np.asarray(dens, float), np.asarray(emit, float).reshape(-1, 3), **kw)


def gauss_depth(o, d, t_end, mu, s, kappa):
    """Optical depth of one Gaussian blob along o + t d, t in [0, t_end] (erf closed form)."""
    f = np.asarray(o, float) - np.asarray(mu, float)
    b = float(f @ d)
    perp = float(f @ f) - b * b
    a = math.sqrt(2.0) * s
    return kappa * math.exp(-perp / (2 * s * s)) * s * math.sqrt(math.pi / 2) * (
        math.erf((t_end + b) / a) - math.erf(b / a))


def bg(v, d):
    w = 0.5 * (1.0 + d[2])
    return np.asarray(v.bg0) + np.asarray(v.bg1) * w


def chord(M, N, i, j):
    p, q = oracle.sf_point(M, i), oracle.sf_point(N, j)
    d = q - p
    return p, q, d / np.linalg.norm(d)


def test_empty_volume_is_background():
    v = vol(np.zeros((0, 3)), [], [], np.zeros((0, 3)))
    M, N = 64, 32
    T = oracle.volume_table(v, M, N, 4)
    for i, j in [(0, 0), (5, 17), (63, 31), (30, 2)]:
        _, _, d = chord(M, N, i, j)
        np.testing.assert_allclose(T[i, j, :3], bg(v, d), rtol=0, atol=1e-7)
        assert T[i, j, 3] == 0.0


def test_segment_ends_at_the_direction_point():
    # Unjittered r_k starts at O + R p_i and leaves S exactly at O + R p_j: t_end = R |p_j - p_i|.
    v = vol([[0, 0, 0]], [0.2], [1.0], [[1, 1, 1]], R=2.5, O=(0.3, -0.2, 0.1))
    M, N = 200, 50
    for i, j in [(3, 7), (100, 25), (199, 0), (57, 49)]:
        p, q, d = chord(M, N, i, j)
        o = oracle.volume_origin(v, M, N, i, j, 0)
        np.testing.assert_allclose(o, np.asarray(v.O) + v.R * p, rtol=0, atol=1e-15)
        _, _, t_end = oracle.volume_ray(v, o, d)
        assert abs(t_end - v.R * np.linalg.norm(q - p)) < 1e-12


@pytest.mark.parametrize("R,O", [(1.0, (0.0, 0.0, 0.0)), (3.0, (1.0, -2.0, 0.5))])
def test_single_blob_closed_form(R, O):
    # With emission = density x colour, L = e (1 - e^-tau) + e^-tau bg exactly; the midpoint
    # rule is exact per step, so only the quadrature of tau is approximated.
    mu = np.asarray(O) + R * np.array([0.1, -0.2, 0.15])
    e = np.array([0.9, 0.4, 0.2])
    v = vol([mu], [0.2 * R], [5.0 / R], [e], steps=20000, R=R, O=O)
    M, N = 128, 64
    for i, j in [(10, 40), (64, 3), (90, 60), (127, 31)]:
        _, _, d = chord(M, N, i, j)
        o = oracle.volume_origin(v, M, N, i, j, 0)
        rgb, T, t_end = oracle.volume_ray(v, o, d)
        tau = gauss_depth(o, d, t_end, mu, 0.2 * R, 5.0 / R)
        assert abs(T - math.exp(-tau)) < 1e-9
        np.testing.assert_allclose(rgb, e * (1 - math.exp(-tau)) + math.exp(-tau) * bg(v, d),
                                   rtol=0, atol=1e-9)


def test_two_blobs_same_colour_add_depths():
    e = np.array([0.3, 0.8, 0.5])
    mus = [[0.2, 0.1, 0.0], [-0.25, 0.0, 0.2]]
    v = vol(mus, [0.15, 0.3], [8.0, 3.0], [e, e], steps=20000)
    M, N = 128, 64
    for i, j in [(20, 50), (70, 10)]:
        _, _, d = chord(M, N, i, j)
        o = oracle.volume_origin(v, M, N, i, j, 0)
        rgb, T, t_end = oracle.volume_ray(v, o, d)
        tau = sum(gauss_depth(o, d, t_end, m, s, k) for m, s, k in zip(mus, [0.15, 0.3], [8.0, 3.0]))
        np.testing.assert_allclose(rgb, e * (1 - math.exp(-tau)) + math.exp(-tau) * bg(v, d),
                                   rtol=0, atol=1e-9)


def test_front_blob_occludes_back_blob():
    # Two narrow blobs 20 widths apart on the x axis; the ray enters at x = -1 heading +x.
    # L = e1 (1 - T1) + T1 e2 (1 - T2) + T1 T2 bg, T_b = exp(-kappa_b s_b sqrt(2 pi)).
    e1, e2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    v = vol([[-0.5, 0, 0], [0.5, 0, 0]], [0.05, 0.05], [20.0, 10.0], [e1, e2], steps=20000)
    o, d = np.array([-1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    rgb, T, t_end = oracle.volume_ray(v, o, d)
    assert abs(t_end - 2.0) < 1e-15
    T1 = math.exp(-20.0 * 0.05 * math.sqrt(2 * math.pi))
    T2 = math.exp(-10.0 * 0.05 * math.sqrt(2 * math.pi))
    want = e1 * (1 - T1) + T1 * e2 * (1 - T2) + T1 * T2 * bg(v, d)
    np.testing.assert_allclose(rgb, want, rtol=0, atol=1e-9)
    assert abs(T - T1 * T2) < 1e-12
    # and from the other side the order is reversed
    rgb2, _, _ = oracle.volume_ray(v, -o, -d)
    want2 = e2 * (1 - T2) + T2 * e1 * (1 - T1) + T1 * T2 * bg(v, -d)
    np.testing.assert_allclose(rgb2, want2, rtol=0, atol=1e-9)


def test_midpoint_rule_is_second_order():
    # A wide blob centred near the entry point, cut off by the segment's ends (a blob that
    # vanishes at both ends would make the midpoint rule converge faster than any power).
    mu, s, k = [-0.8, 0.1, 0.0], 0.4, 0.5
    e = np.array([1.0, 1.0, 1.0])
    o, d = np.array([-1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0])
    errs = []
    for steps in (16, 64):
        v = vol([mu], [s], [k], [e], steps=steps)
        _, T, t_end = oracle.volume_ray(v, o, d)
        errs.append(abs(T - math.exp(-gauss_depth(o, d, t_end, mu, s, k))))
    ratio = errs[0] / errs[1]
    assert 14.0 < ratio < 18.0, ratio     # 16 for O(dt^2); a one-sided rule gives 4


def test_jitter_disk_geometry_and_distribution():
    M, N = 1024, 64
    v = vol([[0, 0, 0]], [0.2], [1.0], [[1, 1, 1]], spp=64, jitter=1, seed=11, R=2.0, O=(0.5, 0.0, -1.0))
    rd = 2.0 * v.R / math.sqrt(M)            # disk of area 4 pi R^2 / M
    offs = []
    for i, j in [(0, 0), (300, 7), (511, 63), (1023, 31)]:
        p = oracle.sf_point(M, i)
        for s in range(v.spp):
            o = oracle.volume_origin(v, M, N, i, j, s)
            off = o - np.asarray(v.O) - v.R * p
            assert abs(off @ p) < 1e-14             # tangent plane at O + R p
            assert np.linalg.norm(off) <= rd * (1 + 1e-12)
            offs.append(off / rd)
    offs = np.array(offs)
    r2 = (offs ** 2).sum(1)
    # uniform on the disk: E[r^2] = 1/2 of the radius squared, half the samples inside r/sqrt(2)
    assert abs(r2.mean() - 0.5) < 0.06
    assert abs((r2 <= 0.5).mean() - 0.5) < 0.1
    # a different texel or sample draws a different point
    a = oracle.volume_origin(v, M, N, 300, 7, 0)
    b = oracle.volume_origin(v, M, N, 300, 7, 1)
    c = oracle.volume_origin(v, M, N, 300, 8, 0)
    assert np.linalg.norm(a - b) > 0 and np.linalg.norm(a - c) > 0


def test_texel_is_the_mean_of_its_samples_and_opacity():
    v = lf_inputs.draw_volume(3, B=5, spp=6, steps=40)
    M, N = 256, 64
    i, j = 77, 40
    _, _, d = chord(M, N, i, j)
    rgbs, ops = [], []
    for s in range(v.spp):
        o = oracle.volume_origin(v, M, N, i, j, s)
        rgb, T, _ = oracle.volume_ray(v, o, d)
        rgbs.append(rgb)
        ops.append(1 - T)
    got = oracle.volume_table(v, M, N, 4, texels=[[i, j]])[0]
    np.testing.assert_allclose(got[:3], np.mean(rgbs, 0), rtol=0, atol=1e-15)
    assert abs(got[3] - np.mean(ops)) < 1e-15


def test_scale_invariance():
    # Scaling lengths by lam and densities by 1/lam leaves every optical depth and radiance
    # unchanged (a dropped factor of R or dt would not).
    base = lf_inputs.draw_volume(5, B=4, spp=3, steps=48)
    lam, O = 3.5, np.array([2.0, -1.0, 0.25])
    big = lf_inputs.Volume(O + lam * (base.mu - np.asarray(base.O)), lam * base.width, base.dens / lam,
                           base.emit, spp=base.spp, steps=base.steps, jitter=base.jitter,
                           seed=base.seed, R=lam * base.R, O=tuple(O))
    M, N = 128, 64
    tex = np.array([[3, 5], [64, 60], [100, 1], [127, 33]])
    np.testing.assert_allclose(oracle.volume_table(big, M, N, 4, texels=tex),
                               oracle.volume_table(base, M, N, 4, texels=tex), rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------------------
# Direct render of the volume (the ground truth of a light-field render)
# --------------------------------------------------------------------------
def _views():
    return lf_inputs.pack_offsets([lf_inputs.look_at((2.5, 0.3, 0.2), (0, 0, 0), 40, 30),
                                   lf_inputs.look_at((0.2, -0.1, -3.0), (0.1, 0, 0), 24, 24)])


def test_direct_pixels_of_an_empty_volume_are_the_background():
    v = vol(np.zeros((0, 3)), [], [], np.zeros((0, 3)))
    views = _views()
    pix = lf_inputs.pixel_list(views)
    out, hits = oracle.volume_pixels(v, views, pix)
    n_hit = 0
    for k, (vi, x, y) in enumerate(pix):
        hit, d, _, _, _, _ = oracle.trace_pixel(1.0, (0, 0, 0), views[vi], x, y)
        if hit:
            n_hit += 1
            np.testing.assert_allclose(out[k, :3], bg(v, d.astype(float)), rtol=0, atol=1e-15)
            assert out[k, 3] == 0.0
        else:
            assert np.all(out[k] == 0.0)
    assert hits == n_hit > 100


def test_direct_pixel_single_blob_closed_form():
    # The pixel's ray enters S at h_o and leaves at h_d: tau from the erf closed form
    # over [0, |h_d - h_o|] (the FP32 hits are within ~1e-7 of the exact chord ends).
    mu = np.array([0.1, -0.2, 0.15])
    e = np.array([0.9, 0.4, 0.2])
    v = vol([mu], [0.2], [5.0], [e], steps=20000)
    views = _views()
    pix = lf_inputs.pixel_list(views, stride=7)
    out, hits = oracle.volume_pixels(v, views, pix)
    checked = 0
    for k, (vi, x, y) in enumerate(pix):
        hit, d, ho, hd, _, _ = oracle.trace_pixel(1.0, (0, 0, 0), views[vi], x, y)
        if not hit:
            continue
        d = d.astype(float)
        tau = gauss_depth(ho.astype(float), d, float(np.linalg.norm(hd.astype(float) - ho)), mu, 0.2, 5.0)
        want = e * (1 - math.exp(-tau)) + math.exp(-tau) * bg(v, d)
        np.testing.assert_allclose(out[k, :3], want, rtol=0, atol=2e-6)
        assert abs(out[k, 3] - (1 - math.exp(-tau))) < 2e-6
        checked += 1
    assert checked > 20


def test_direct_pixel_along_a_chord_equals_the_unjittered_texel():
    # A single-pixel view aimed from outside S through O + R p_i at O + R p_j sees the
    # ray r_k of texel (i, j) without jitter: the same radiance up to the FP32 rounding
    # of its front hit.
    v = lf_inputs.draw_volume(4, B=6, spp=1, steps=48)
    v.jitter = 0
    M, N = 300, 120
    rng = np.random.default_rng(3)
    pairs = [(int(rng.integers(M)), int(rng.integers(N))) for _ in range(60)]
    views = []
    for i, j in pairs:
        p, q, d = chord(M, N, i, j)
        views.append(lf_inputs.look_at(p - rng.uniform(0.3, 2.0) * d, q, 1, 1))
    views = lf_inputs.pack_offsets(views)
    out, hits = oracle.volume_pixels(v, views, lf_inputs.pixel_list(views))
    want = oracle.volume_table(v, M, N, 4, texels=np.array(pairs))
    assert hits == len(pairs)
    np.testing.assert_allclose(out, want, rtol=0, atol=3e-6)


def test_light_field_render_converges_to_the_direct_render():
    # The light-field render of the precomputed table approaches the direct render of
    # the volume as the SF sets grow (Section 2: the table samples the rays between the
    # two point sets; the filter blends the nearest ones): PSNR rises with M and N.
    v = lf_inputs.draw_volume(8, B=8, spp=2, steps=32)
    views = [lf_inputs.look_at(np.array([2.1, -1.3, 0.8]), (0, 0, 0), 96, 72)]
    gt, hits = oracle.volume_pixels(v, views, lf_inputs.pixel_list(views))
    psnr = []
    for M, N in [(256, 64), (1024, 256), (4096, 512)]:
        T = oracle.volume_table(v, M, N, 4)
        out, idx, _ = oracle.render_views(oracle.Scene(M, N, 4, "f32", T), views)
        hit = idx[:, 0] >= 0
        assert hit.sum() == hits > 3000
        psnr.append(oracle.psnr(gt[:, :3], out[:, :3], hit))
    assert psnr[0] > 25 and psnr[1] > psnr[0] + 4 and psnr[2] > psnr[1] + 4, psnr


def test_direct_pixel_along_a_chord_of_a_moved_sphere():
    # the same correspondence for S of radius 2.5 centred away from the origin
    v = lf_inputs.draw_volume(5, B=5, spp=1, steps=40, R=2.5, O=(0.5, -0.25, 1.0))
    v.jitter = 0
    M, N = 200, 90
    O = np.asarray(v.O)
    rng = np.random.default_rng(6)
    pairs = [(int(rng.integers(M)), int(rng.integers(N))) for _ in range(40)]
    views = []
    for i, j in pairs:
        p, q, d = chord(M, N, i, j)
        a, b = O + v.R * p, O + v.R * q
        views.append(lf_inputs.look_at(a - rng.uniform(0.5, 4.0) * d, b, 1, 1))
    views = lf_inputs.pack_offsets(views)
    out, hits = oracle.volume_pixels(v, views, lf_inputs.pixel_list(views))
    want = oracle.volume_table(v, M, N, 4, texels=np.array(pairs))
    assert hits == len(pairs)
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-5)
