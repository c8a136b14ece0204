"""Stored expected values (tests/golden/, written by make_golden.py from the oracle alone): the
oracle still reproduces them, and the CUDA path matches them (config 1, GPU part marked)."""
import os

import numpy as np
import pytest

from tests.golden.make_golden import config1_values, read

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_q2_8cubed.txt")


def test_oracle_reproduces_stored_config1(oracle):
    stored = read(GOLDEN)
    fresh = config1_values()
    for key in ("y_sample", "y_sum", "y_maxabs", "cg_history", "x50_sample"):
        ref = stored[key]
        assert np.abs(fresh[key] - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300), key
    # the history is the relative residual of a convergent CG: starts at 1, ends far lower
    assert stored["cg_history"][0] == 1.0 and stored["cg_history"][-1] < 1e-6


@pytest.mark.gpu
def test_cuda_path_matches_stored_config1():
    import torch

    import paper_2609_04534_gb300 as mf
    from paper_2609_04534_gb300 import inputs
    from tests._gpu import DevOp

    stored = read(GOLDEN)
    N, k = 8, 2
    x = inputs.random_unique(N, N, N, k, 0)
    d0 = DevOp(N, N, N, k, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    y = d0.unique_from_native(d0.apply(d0.native_from_unique(x)))
    idx = stored["y_index"].astype(int)
    assert np.abs(y[idx] - stored["y_sample"]).max() <= 1e-12 * stored["y_maxabs"][0]
    d0.close()
    d1 = DevOp(N, N, N, k, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 1)
    xt = x.copy()
    # boundary nodes of the 17^3 node lattice
    I = np.arange(d1.n_unique)
    n1 = N * k + 1
    i, j, l = I % n1, (I // n1) % n1, I // (n1 * n1)
    mask = (i == 0) | (i == n1 - 1) | (j == 0) | (j == n1 - 1) | (l == 0) | (l == n1 - 1)
    xt[mask] = 0.0
    b = d1.apply(d1.native_from_unique(xt))
    xs = torch.zeros(d1.n_native, dtype=torch.float64, device="cuda")
    ws = torch.empty(mf.mf_cg_workspace_bytes(d1.op, 0), dtype=torch.uint8, device="cuda")
    hist = np.zeros(64)
    mf.mf_cg_record_history(hist.ctypes.data, 64)
    try:
        st = mf.mf_cg_solve(d1.op, b.data_ptr(), xs.data_ptr(), 0.0, 50, 0, ws.data_ptr(), ws.numel(),
                            allow_not_converged=True)
    finally:
        mf.mf_cg_record_history(None, 0)
    assert st["iterations"] == 50
    np.testing.assert_allclose(hist[:51], stored["cg_history"], rtol=1e-10, atol=0)
    xg = d1.unique_from_native(xs)
    ix = stored["x50_index"].astype(int)
    assert np.abs(xg[ix] - stored["x50_sample"]).max() <= 1e-10 * np.abs(stored["x50_sample"]).max()
    d1.close()
