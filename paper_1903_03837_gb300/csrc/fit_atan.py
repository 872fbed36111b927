"""Coefficients of the azimuth polynomial in lf_device.cuh (azimuth_turns).

atan(a) for a in [0, 1] is approximated by the odd polynomial
a * (c0 + c1 a^2 + ... + c7 a^14) (degree 15). The coefficients minimise the
largest absolute error over [0, 1] (minimax), found by Lawson's algorithm:
weighted least squares on Chebyshev nodes of [0, 1], each weight multiplied
by the node's current absolute error and renormalised, until the weights
settle (C. L. Lawson, "Contributions to the theory of linear least maximum
approximation", 1961). The result is rounded to float32.

  python fit_atan.py            # prints the float32 coefficients
"""
import numpy as np

DEGREE_TERMS = 8          # c0 .. c7: odd degree 15
NODES = 4000
ITERATIONS = 400


def fit(terms: int = DEGREE_TERMS, nodes: int = NODES, iterations: int = ITERATIONS) -> np.ndarray:
    k = np.arange(nodes)
    a = 0.5 + 0.5 * np.cos(np.pi * (2 * k + 1) / (2 * nodes))       # Chebyshev nodes of [0, 1]
    A = a[:, None] * (a * a)[:, None] ** np.arange(terms)[None, :]
    y = np.arctan(a)
    w = np.full(nodes, 1.0 / nodes)
    c = None
    for _ in range(iterations):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y)
        w = w * e
        w /= w.sum()
    return c


def coefficients_f32() -> np.ndarray:
    return fit().astype(np.float32)


def eval_f32(c: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Horner in float32 with one rounding per multiply-add, as the kernel's
    __fmaf_rn chain (exact product and sum in float64, rounded once: exact for
    float32 operands up to a double rounding that is far below the fit error)."""
    a = a.astype(np.float32)
    a2 = (a * a).astype(np.float32)
    p = np.full_like(a, c[-1])
    for ck in c[-2::-1]:
        p = (p.astype(np.float64) * a2.astype(np.float64) + np.float64(ck)).astype(np.float32)
    return (a * p).astype(np.float32)


if __name__ == "__main__":
    c = coefficients_f32()
    print(", ".join(repr(float(x)) + "f" for x in c))
    a = np.linspace(0.0, 1.0, 1_000_001)
    print("max |error| in float32 evaluation:", float(np.abs(eval_f32(c, a).astype(np.float64) - np.arctan(a)).max()))
