"""Writes kernel_size.txt: the paper's printed kernel-size expression (Section 2),
R * 5^(1/4) * sqrt(4*pi/(sqrt(5)*N)), evaluated in 50-digit arithmetic. Calls
no code of this repository."""
import os

import mpmath

mpmath.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))
rows = [(1.0, 256), (1.0, 1024), (1.0, 4096), (2.5, 512), (1.0, 16384), (1.0, 23576),
        (0.75, 65536), (1.0, 262144)]
with open(os.path.join(HERE, "kernel_size.txt")) as f:
    head = [ln for ln in f if ln.startswith("#")]
with open(os.path.join(HERE, "kernel_size.txt"), "w") as f:
    f.writelines(head)
    for R, N in rows:
        v = mpmath.mpf(R) * mpmath.root(5, 4) * mpmath.sqrt(4 * mpmath.pi / (mpmath.sqrt(5) * N))
        f.write(f"{R} {N} {mpmath.nstr(v, 25)}\n")
