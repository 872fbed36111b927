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


def test_select7_of16_keeps_the_seven_smallest_sorted():
    net = _network("void select7_of16")
    assert len(net) == 54
    assert _sorts_prefix(net, 16, 7)


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
