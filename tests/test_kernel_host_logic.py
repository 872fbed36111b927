"""Host-side checks of logic that the CUDA kernels hard-code: the comparator
networks of the K-NN selection (0-1 principle over every binary input) and
the Fibonacci / lattice-offset table (Binet closed form)."""
import itertools
import math
import os
import re

import pytest

from paper_1903_03837_gb300 import build as B

DEV = os.path.join(B.CSRC, "lf_device.cuh")


def _network(fn_name):
    src = open(DEV).read()
    body = src[src.index(fn_name):]
    body = body[body.index("{") + 1: body.index("\n}")]
    return [(int(a), int(b)) for a, b in re.findall(r"LF_CS\((\d+),\s*(\d+)\)", body)]


def _sorts_prefix(net, n, k):
    for m in range(1 << n):
        v = [(m >> i) & 1 for i in range(n)]
        for a, b in net:
            if v[a] > v[b]:
                v[a], v[b] = v[b], v[a]
        if v[:k] != sorted(v)[:k]:
            return False
    return True


def test_select7_of12_keeps_the_seven_smallest_sorted():
    net = _network("void select7_of12")
    assert len(net) == 37
    assert all(0 <= a < b < 12 for a, b in net)
    assert _sorts_prefix(net, 12, 7)


def _sorts_prefix_packed(net, n, k):
    """The 0-1 principle over all 2^n binary inputs, 64 inputs per machine
    word: line i holds bit i of every input index; a comparator is AND (min)
    and OR (max); output m must be 1 exactly for the inputs with at most m
    zeros."""
    import numpy as np
    idx = np.arange(1 << n, dtype=np.uint32)
    lines = [np.packbits(((idx >> i) & 1).astype(np.uint8), bitorder="little").view(np.uint64) for i in range(n)]
    for a, b in net:
        lines[a], lines[b] = lines[a] & lines[b], lines[a] | lines[b]
    zeros = n - np.bitwise_count(idx).astype(np.int64)
    for m in range(k):
        want = np.packbits((zeros <= m).astype(np.uint8), bitorder="little").view(np.uint64)
        if not np.array_equal(lines[m], want):
            return False
    return True


def test_select10_of25_keeps_the_ten_smallest_sorted():
    net = _network("void select10_of25")
    assert len(net) == 119
    assert all(0 <= a < b < 25 for a, b in net)
    assert _sorts_prefix_packed(net, 25, 10)


def test_packed_check_rejects_a_broken_network():
    net = _network("void select10_of25")
    assert not _sorts_prefix_packed(net[:-1], 25, 10)


def test_sort6_sorts():
    net = _network("void sort6")
    assert len(net) == 12
    assert _sorts_prefix(net, 6, 6)


def test_lattice_offsets_follow_binet():
    # eps_k = F_k / Phi - F_{k-1} = (-1)^(k+1) Phi^-k: the lattice basis of SF points
    phi = (1 + 5 ** 0.5) / 2
    F = [0, 1]
    while len(F) < 40:
        F.append(F[-1] + F[-2])
    for k in range(1, 38):
        eps = F[k] / phi - F[k - 1]
        assert abs(eps - (-1) ** (k + 1) * phi ** (-k)) < 1e-9 * max(1.0, F[k])
        # the basis (eps_k, F_k), (eps_{k+1}, F_{k+1}) has determinant
        # eps_k F_{k+1} - eps_{k+1} F_k = F_k^2 - F_{k-1} F_{k+1} = (-1)^(k+1) (Cassini): unimodular
        assert F[k] * F[k] - F[k - 1] * F[k + 1] == (-1) ** (k + 1)


def _kernel_atan_coefficients():
    import numpy as np
    src = open(DEV).read()
    body = src[src.index("kAtanC[8] = {") + len("kAtanC[8] = {"):]
    body = body[:body.index("}")]
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")], dtype=np.float32)


def test_azimuth_coefficients_come_from_the_fit_script():
    """The kernel's atan coefficients are those fit_atan.py writes (minimax by
    Lawson's algorithm, rounded to float32)."""
    import importlib.util
    import numpy as np
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(B.CSRC, "fit_atan.py"))
    fit = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fit)
    c = _kernel_atan_coefficients()
    assert len(c) == 8
    assert np.array_equal(c, fit.coefficients_f32())
    # the fit in exact arithmetic is minimax-small, and float32 Horner stays near it
    a = np.linspace(0.0, 1.0, 200001)
    assert np.abs(a * np.polyval(fit.fit()[::-1], a * a) - np.arctan(a)).max() < 5e-8
    assert np.abs(fit.eval_f32(c, a).astype(np.float64) - np.arctan(a)).max() < 2e-7


def test_azimuth_polynomial_accuracy():
    """The kernel's azimuth, evaluated in float32 as the kernel does (quotient,
    polynomial, the pi/2 and pi reflections, each rounded), stays within 5e-7
    rad of atan2 on random points of all four quadrants (the lattice window
    tolerates 2e-3 cells, i.e. about 1.9e-6 rad for the largest Fibonacci step
    of n = 2^24 points)."""
    import numpy as np
    c = _kernel_atan_coefficients()
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 200000)
    rad = rng.uniform(1e-3, 1.0, 200000)
    x = (rad * np.cos(ang)).astype(np.float32)
    y = (rad * np.sin(ang)).astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    a = (np.minimum(ax, ay) / np.maximum(ax, ay)).astype(np.float32)
    a2 = (a * a).astype(np.float32)
    p = np.full_like(a, c[7])
    for k in range(6, -1, -1):
        p = (p.astype(np.float64) * a2 + np.float64(c[k])).astype(np.float32)
    r = (a * p).astype(np.float32)
    r = np.where(ay > ax, np.float32(1.57079632679) - r, r)
    r = np.where(x < 0, np.float32(3.14159265359) - r, r)
    r = np.where(y < 0, -r, r)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    d = np.abs(np.angle(np.exp(1j * (r.astype(np.float64) - ref))))
    assert d.max() < 5e-7
