"""Writes the stored expected values under tests/golden/ from the CPU oracle alone.

Config 1 of the benchmark definition: Q2 Laplace on the affine unit cube, 8^3 cells, FP64,
x uniform[-1, 1] from the seed-0 splitmix64 stream on unique DoFs.  Stored:
  * y = A x without boundary conditions (every 61st unique DoF, plus the sum and the max-norm),
  * 50 CG iterations on P A P x = b with b = P A P x_true, x_true = the seed-0 vector masked at
    the boundary (the relative residual history, and every 61st entry of x_50).
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_04534_gb300 import inputs  # noqa: E402  (seeded generator only)

STRIDE = 61


def config1_values():
    N, k = 8, 2
    o0 = oracle.Op(N, N, N, k, oracle.AFFINE, bc=0)
    x = inputs.random_unique(N, N, N, k, 0)
    y = o0.apply(x, nthreads=1)
    o1 = oracle.Op(N, N, N, k, oracle.AFFINE, bc=1)
    xt = x.copy()
    xt[o1.boundary_mask()] = 0.0
    b = o1.apply(xt, nthreads=1)
    x50, hist = o1.cg(b, maxit=50, rtol=0.0, nthreads=1)
    return {
        "y_index": np.arange(0, y.size, STRIDE),
        "y_sample": y[::STRIDE],
        "y_sum": np.array([y.sum()]),
        "y_maxabs": np.array([np.abs(y).max()]),
        "cg_history": hist,
        "x50_index": np.arange(0, x50.size, STRIDE),
        "x50_sample": x50[::STRIDE],
    }


def write(path, values):
    with open(path, "w") as f:
        f.write("# Written by tests/golden/make_golden.py from the CPU oracle alone (no CUDA path).\n")
        f.write("# Config 1: Q2 Laplace, affine unit cube, 8^3 cells, FP64, seed-0 x on unique DoFs;\n")
        f.write("# y = A x without boundary conditions, and 50 CG iterations with homogeneous Dirichlet.\n")
        for key, arr in values.items():
            f.write(f"{key} " + " ".join(repr(float(v)) if arr.dtype.kind == "f" else str(int(v)) for v in arr) + "\n")


def read(path):
    out = {}
    with open(path) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            key, *vals = ln.split()
            out[key] = np.array([float(v) for v in vals])
    return out


if __name__ == "__main__":
    oracle.build()
    write(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_q2_8cubed.txt"), config1_values())
    print("written")
