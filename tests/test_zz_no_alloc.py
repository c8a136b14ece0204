"""mf_dot_noalloc: the reduction for callers that may not allocate device memory (its
scratch is a static array inside libmf).  It must agree with mf_dot (which takes caller
scratch) within the dot-product tolerance of the other tests, on two calls in a row, and
reject vectors longer than its static scratch supports.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._gpu import DevOp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,dims,k", [(mf.MF_FP64, (5, 6, 3), 3), (mf.MF_FP32, (5, 6, 3), 3),
                                         (mf.MF_FP64, (40, 40, 40), 4)])
def test_noalloc_dot_matches_mf_dot_twice(prec, dims, k):
    d = DevOp(*dims, k, "curved", mf.MF_HELMHOLTZ, 1.0, prec, 0)
    a = inputs.random_unique(*dims, k, 31)
    b = inputs.random_unique(*dims, k, 32)
    an, bn = d.native_from_unique(a), d.native_from_unique(b)
    ys = d.apply(an, split=True)
    for split, u, v in ((0, an, bn), (1, ys, bn)):
        ref = d.dot(u, v, split=split)
        bound = 1e-13 * float((u.double().abs() * v.double().abs()).sum())
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            mf.mf_dot_noalloc(d.op, u.data_ptr(), v.data_ptr(), out.data_ptr(), split)
            torch.cuda.synchronize()
            got = float(out.item())
            assert np.isfinite(got)
            assert abs(got - ref) <= bound, (split, got, ref)
    d.close()


def test_noalloc_dot_rejects_vectors_beyond_its_static_scratch():
    mesh = mf.mf_mesh_create(256, 256, 128)
    op = mf.mf_operator_create(mesh, 3)
    assert mf.mf_operator_info(op)["n_native"] > 134_217_728
    with pytest.raises(mf.MfError) as e:
        mf.mf_dot_noalloc(op, 256, 512, 1024)  # rejected before any device access
    assert e.value.code == mf.MF_ERR_ARG
    assert "limit" in str(e.value)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)
