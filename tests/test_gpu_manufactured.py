"""GPU manufactured-solution kernels (right-hand side and L2 error) against the oracle, and a
mixed-precision solve of the manufactured Poisson problem converging at rate k+1."""
import math

import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from tests._fem_ref import solve_direct
from tests._gpu import DevOp, oracle_op, rel_max

pytestmark = pytest.mark.gpu


def scratch_for(d):
    return torch.empty(mf.mf_manufactured_workspace_bytes(d.op), dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("k", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("geom,kind,bc,prec", [("curved", mf.MF_LAPLACE, 1, mf.MF_FP64),
                                                ("cart", mf.MF_HELMHOLTZ, 0, mf.MF_FP64),
                                                ("stretch", mf.MF_LAPLACE, 1, mf.MF_FP64),
                                                ("curved", mf.MF_HELMHOLTZ, 0, mf.MF_FP32)])
def test_rhs_matches_oracle(oracle, k, geom, kind, bc, prec):
    dims = (5, 4, 3)
    freq = 2.0
    d = DevOp(*dims, k, geom, kind, 1.0, prec, bc)
    o = oracle_op(oracle, *dims, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
    b = torch.full((d.n_native,), float("nan"), dtype=d.dtype, device="cuda")
    sc = scratch_for(d)
    mf.mf_rhs_manufactured(d.op, freq, b.data_ptr(), sc.data_ptr(), sc.numel())
    got = d.unique_from_native(b)
    ref = o.rhs_manufactured(freq, nqr=k + 1)
    # scale from the unmasked load vector: on some meshes every free entry vanishes by symmetry
    scale = np.abs(ref).max()
    if bc:
        ref[o.boundary_mask()] = 0.0
    tol = 1e-12 if prec != mf.MF_FP32 else 1e-6
    assert np.abs(got - ref).max() <= tol * scale
    # consistent: every copy equal
    assert torch.equal(d.native_from_unique(got), b.double().to(d.dtype)) or prec == mf.MF_FP32
    d.close()


@pytest.mark.parametrize("k,geom", [(2, "curved"), (3, "cart"), (5, "curved")])
def test_l2_error_matches_oracle(oracle, k, geom):
    dims, freq = (4, 3, 5), 2.0
    d = DevOp(*dims, k, geom, mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    o = oracle_op(oracle, *dims, k, geom, 0.0, 0)
    uh = o.interpolate_manufactured(freq) * 0.97 + 0.01  # not the exact interpolant
    un = d.native_from_unique(uh)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sc = scratch_for(d)
    mf.mf_error_manufactured(d.op, freq, un.data_ptr(), out.data_ptr(), sc.data_ptr(), sc.numel())
    torch.cuda.synchronize()
    l2_ref, _ = o.errors(uh, freq, nqr=k + 1)
    assert abs(math.sqrt(out.item()) - l2_ref) <= 1e-12 * l2_ref
    d.close()


@pytest.mark.parametrize("k", [2, 3])
def test_mixed_solve_manufactured_converges(oracle, k):
    """Mixed-precision solve of -Lap u = f on the curved mesh; L2 error falls at rate ~k+1 and
    matches the oracle's direct FP64 solution error."""
    errs = []
    for N in (4, 8):
        d = DevOp(N, N, N, k, "curved", mf.MF_LAPLACE, 1.0, mf.MF_MIXED, 1)
        b = torch.empty(d.n_native, dtype=torch.float64, device="cuda")
        sc = scratch_for(d)
        mf.mf_rhs_manufactured(d.op, 2.0, b.data_ptr(), sc.data_ptr(), sc.numel())
        x = torch.zeros_like(b)
        ws = torch.empty(mf.mf_cg_workspace_bytes(d.op, 1), dtype=torch.uint8, device="cuda")
        st = mf.mf_cg_solve(d.op, b.data_ptr(), x.data_ptr(), 1e-10, 20000, 1, ws.data_ptr(), ws.numel())
        assert st["rel_residual"] <= 1e-10
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        mf.mf_error_manufactured(d.op, 2.0, x.data_ptr(), out.data_ptr(), sc.data_ptr(), sc.numel())
        torch.cuda.synchronize()
        errs.append(math.sqrt(out.item()))
        o = oracle_op(oracle, N, N, N, k, "curved", 0.0, 1)
        xo = solve_direct(o, o.rhs_manufactured(2.0, nqr=k + 1))
        l2o, _ = o.errors(xo, 2.0, nqr=k + 1)
        assert abs(errs[-1] - l2o) <= 1e-6 * l2o
        d.close()
    rate = math.log2(errs[0] / errs[1])
    assert rate > k + 0.5, (errs, rate)
