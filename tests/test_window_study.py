"""Completeness of the inverse-SF lattice windows (Section 2: Keinert's inverse
mapping extended to the 5, and up to 9, nearest points).

The render kernels never search the whole point set. Away from the poles they
rank the 12 lattice corners of `lattice_window` (5 neighbours) or the 5x5
block around the rounded corner (9 neighbours); within 16 continuous indices
of a pole they scan the 64 points nearest that pole. Their tier-1/tier-2
certificates prove the *order* of the candidates, not that the true nearest
points are among them. This file is that second proof, by brute force: for
n = 256 ... 2^24 points and 10^6 random queries per n, the true nearest points
(a k-d tree over the FP64 points) must lie inside the window.

The window is restated here from the kernel's construction (zone k, Fibonacci
pair, lattice coordinates (u, v) in the basis (eps_k, F_k), (eps_{k+1},
F_{k+1}), the rounded corner, the sign quadrant, and the quadrant's quarter
turn of the basis) in FP64. The kernel computes (u, v) in FP32; its error is
below 7e-4 cells for n <= 2^24: the float32 azimuth is within 5e-7 rad of
atan2 (tests/test_kernel_host_logic.py), i.e. 8e-8 turns, times F_{k+1} <=
6765 gives 5.4e-4 cells; the turn conversion and the multiply-adds add about
1e-4; the continuous index, up to 1 index unit for n = 2^24, times |eps| <=
7e-5. Every query is therefore checked with (u, v) moved by -2e-3, 0 and +2e-3
cells in all nine combinations, and with the zone's continuous value moved by
+-0.02 (which flips the zone of queries next to a zone boundary).
"""
import functools
import math

import numpy as np
import pytest

import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")

PHI = (1.0 + 5.0 ** 0.5) / 2.0
_F = [0, 1]
while len(_F) < 40:
    _F.append(_F[-1] + _F[-2])
F = np.array(_F, dtype=np.int64)
F32 = F.astype(np.int32)
EPS = np.array([(1.0 if k % 2 == 1 else -1.0) * PHI ** (-k) for k in range(40)])   # (-1)^(k+1) Phi^-k

# the 12 window offsets (du, dv) of the quadrant (+,+) in the basis (G0, G1); the
# other quadrants turn the basis: (-,-) (-F0,-F1), (+,-) (-F1,F0), (-,+) (F1,-F0)
WIN12 = np.array([(du, dv) for dv in (-1, 0, 1) for du in (-1, 0, 1)] + [(1, 2), (2, -1), (2, 0)], dtype=np.int32)
WIN25 = np.array([(du, dv) for du in range(-2, 3) for dv in range(-2, 3)], dtype=np.int32)
POLE = 16          # continuous-index distance from a pole below which the kernel scans
POLE_PTS = 64      # points scanned at a pole


def lattice_coords(q, n):
    """Azimuth in turns, continuous index and the zone's continuous value of
    unit queries q (the inputs of the kernel's window, in FP64)."""
    z = q[:, 2]
    t = np.arctan2(q[:, 1], q[:, 0]) / (2.0 * np.pi)
    ic = (n * (1.0 - z) - 1.0) * 0.5
    kc = np.log(math.sqrt(5.0) * math.pi * n * (1.0 - z) * (1.0 + z)) / np.log(PHI * PHI)
    return t, ic, kc


def window_corner(coords, du_off, dv_off, dk):
    """What the kernel's window depends on: the zone k, the rounded corner
    (ru, rv) and the sign quadrant (pu, pv) of the lattice coordinates, here
    moved by (du_off, dv_off) cells and the zone's continuous value by dk."""
    t, ic, kc = coords
    k = np.clip(np.floor(kc + dk).astype(np.int32), 2, 37)
    F0, F1, e0, e1 = F32[k], F32[k + 1], EPS[k], EPS[k + 1]
    sg = np.where(k % 2 == 1, -1.0, 1.0)
    u = sg * (-F1 * t + e1 * ic) + du_off
    v = sg * (F0 * t - e0 * ic) + dv_off
    ru, rv = np.rint(u), np.rint(v)
    return k, ru.astype(np.int32), rv.astype(np.int32), u >= ru, v >= rv


def window_candidates(corner, offsets):
    """Candidate indices [Q, len(offsets)] of the window at `corner` (int32
    throughout: for n <= 2^24 every index and offset is far below 2^31)."""
    k, ru, rv, pu, pv = corner
    F0, F1 = F32[k], F32[k + 1]
    base = ru * F0 + rv * F1
    G0 = np.where(pu, np.where(pv, F0, -F1), np.where(pv, F1, -F0))
    G1 = np.where(pu, np.where(pv, F1, F0), np.where(pv, -F0, -F1))
    return base[:, None] + offsets[None, :, 0] * G0[:, None] + offsets[None, :, 1] * G1[:, None]


def random_queries(rng, count):
    q = rng.normal(size=(count, 3))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def away_from_poles(q, n):
    icn = (n * (1.0 - q[:, 2]) - 1.0) * 0.5
    ics = (n * (1.0 + q[:, 2]) - 1.0) * 0.5
    return (icn >= POLE) & (ics >= POLE)


def missing(cand, nn):
    """Number of queries whose true nearest (rows of nn) are not all in cand."""
    ok = np.ones(len(nn), dtype=bool)
    for j in range(nn.shape[1]):
        ok &= (cand == nn[:, j:j + 1]).any(axis=1)
    return int((~ok).sum())


SIZES = [256, 1000, 4096, 16384, 65536, 262144, 1 << 20, 1 << 22, 1 << 24]


@functools.lru_cache(maxsize=None)
def points_and_tree(n):
    P = oracle.sf_points(n)
    return P, scipy_spatial.cKDTree(P)
QUERIES = 1_000_000


@pytest.mark.parametrize("n", SIZES)
def test_lattice_windows_contain_the_true_nearest(n):
    _, tree = points_and_tree(n)
    rng = np.random.default_rng(n)
    q = random_queries(rng, QUERIES)
    q = q[away_from_poles(q, n)]
    # queries near the poles but outside the pole scan, where the zone is small
    near = random_queries(rng, 400_000)
    near = near[away_from_poles(near, n) & (np.minimum(n * (1 - near[:, 2]), n * (1 + near[:, 2])) < 40 * POLE)]
    q = np.concatenate([q, near])
    _, nn9 = tree.query(q, k=9, workers=-1)
    nn9 = nn9.astype(np.int32)
    nn5 = nn9[:, :5]
    coords = lattice_coords(q, n)
    c0 = window_corner(coords, 0.0, 0.0, 0.0)
    assert missing(window_candidates(c0, WIN12), nn5) == 0, (n, "5 nearest")
    assert missing(window_candidates(c0, WIN25), nn9) == 0, (n, "9 nearest")
    # moved coordinates: only the queries whose corner, quadrant or zone changes
    # get another window; they are checked again
    combos = [(a, b, 0.0) for a in (-2e-3, 0.0, 2e-3) for b in (-2e-3, 0.0, 2e-3) if (a, b) != (0.0, 0.0)]
    combos += [(0.0, 0.0, -0.02), (0.0, 0.0, 0.02)]
    moved = 0
    for du, dv, dk in combos:
        c = window_corner(coords, du, dv, dk)
        diff = np.zeros(len(q), dtype=bool)
        for a, b in zip(c, c0):
            diff |= a != b
        sel = np.nonzero(diff)[0]
        moved += len(sel)
        cs = tuple(a[sel] for a in c)
        assert missing(window_candidates(cs, WIN12), nn5[sel]) == 0, (n, du, dv, dk, "5 nearest")
        assert missing(window_candidates(cs, WIN25), nn9[sel]) == 0, (n, du, dv, dk, "9 nearest")
    assert moved > 1000, moved          # the moves do reach corner, quadrant and zone boundaries


@pytest.mark.parametrize("n", [256, 4096, 262144, 1 << 24])
def test_pole_scans_contain_the_true_nearest(n):
    """Queries within 16 continuous indices of a pole: the 64 points nearest
    that pole (indices 0..63 or n-64..n-1) hold the 5 and the 9 nearest."""
    _, tree = points_and_tree(n)
    rng = np.random.default_rng(7 + n)
    # uniform over the caps of continuous index < 16 (z > 1 - 33/n and the mirror)
    cnt = 200_000
    zc = 1.0 - rng.uniform(0.0, (2 * POLE + 1) / n, cnt)
    ph = rng.uniform(0.0, 2 * np.pi, cnt)
    s = np.sqrt(1.0 - zc * zc)
    north = np.stack([np.cos(ph) * s, np.sin(ph) * s, zc], 1)
    south = north * np.array([1.0, 1.0, -1.0])
    for q, lo in ((north, 0), (south, n - POLE_PTS)):
        inside = ~away_from_poles(q, n)
        q = q[inside]
        assert len(q) > 1000
        _, nn9 = tree.query(q, k=9, workers=-1)
        assert ((nn9 >= lo) & (nn9 < lo + POLE_PTS)).all(), n


def test_window_slots_match_the_kernel_encoding():
    """The kernel numbers the 12 corners by slot s = (du + 1) + 4 (dv + 1):
    s = 0..10 and 14, index b0 + (s & 3) G0 + (s >> 2) G1 with b0 = c - G0 - G1."""
    slots = [j if j < 11 else 14 for j in range(12)]
    dec = sorted(((s & 3) - 1, (s >> 2) - 1) for s in slots)
    assert dec == sorted(map(tuple, WIN12.tolist()))
    # the four quadrant windows are the fixed offsets in the turned bases, and
    # equal the per-quadrant corner lists: 3x3 block plus (-,-): (-2,0) (-1,-2) (-2,1),
    # (-,+): (-2,1) (0,2) (1,2), (+,-): (-1,-2) (0,-2) (2,-1), (+,+): (1,2) (2,-1) (2,0)
    F0, F1 = 13, 21
    ext = {(0, 0): [(-2, 0), (-1, -2), (-2, 1)], (0, 1): [(-2, 1), (0, 2), (1, 2)],
           (1, 0): [(-1, -2), (0, -2), (2, -1)], (1, 1): [(1, 2), (2, -1), (2, 0)]}
    basis = {(1, 1): (F0, F1), (0, 0): (-F0, -F1), (1, 0): (-F1, F0), (0, 1): (F1, -F0)}
    for quad, (G0, G1) in basis.items():
        got = sorted(du * G0 + dv * G1 for du, dv in WIN12.tolist())
        want = sorted([a * F0 + b * F1 for a in (-1, 0, 1) for b in (-1, 0, 1)] + [a * F0 + b * F1 for a, b in ext[quad]])
        assert got == want, quad
