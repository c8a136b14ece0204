"""mf_dot_noalloc: the reduction for callers that may not allocate device memory (its
scratch is a static array inside libmf).  On two calls in a row it must agree with mf_dot
(which takes caller scratch) and with an exactly rounded host sum (math.fsum) of the same
products, within the dot-product tolerance of the other tests.  Collected last on purpose.

The host-side rejections (vectors longer than the static scratch, an operator that was
never set up) are CPU tests in tests/test_lib_abi.py: they must never reach a launch."""
import math

import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._gpu import DevOp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,dims,k", [(mf.MF_FP64, (5, 6, 3), 3), (mf.MF_FP32, (5, 6, 3), 3),
                                         (mf.MF_FP64, (40, 40, 40), 4)])
def test_noalloc_dot_matches_mf_dot_and_fsum_twice(prec, dims, k):
    d = DevOp(*dims, k, "curved", mf.MF_HELMHOLTZ, 1.0, prec, 0)
    a = inputs.random_unique(*dims, k, 31)
    b = inputs.random_unique(*dims, k, 32)
    an, bn = d.native_from_unique(a), d.native_from_unique(b)
    ys = d.apply(an, split=True)
    for split, u, v in ((0, an, bn), (1, ys, bn)):
        if split:  # the pairing of a split dual with a consistent vector: every real copy
            pu, pv = d.canonical_from_native(u), d.canonical_from_native(v)
        else:      # the assembled product: every unique node once
            pu, pv = d.unique_from_native(u), d.unique_from_native(v)
        exact = math.fsum((pu * pv).tolist())
        ref = d.dot(u, v, split=split)
        bound = 1e-13 * float(np.abs(pu * pv).sum())
        assert abs(ref - exact) <= bound, (split, ref, exact)
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            mf.mf_dot_noalloc(d.op, u.data_ptr(), v.data_ptr(), out.data_ptr(), split)
            torch.cuda.synchronize()
            got = float(out.item())
            assert np.isfinite(got)
            assert abs(got - ref) <= bound, (split, got, ref)
            assert abs(got - exact) <= bound, (split, got, exact)
    d.close()
