"""The tensor-core apply of the FP64 Cartesian operator (launch variant MF_VARIANT_TENSOR,
degrees 1..3): parity with the FP64 oracle at 1e-12 (relative max-norm), agreement with the
double-float variants, and the properties its exact digit arithmetic guarantees -- scaling
by a power of two commutes with it bitwise, zeros stay zero, a non-finite value poisons
only its own cell -- plus the device error word staying clear."""
import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._gpu import DevOp, oracle_op, rel_max

pytestmark = pytest.mark.gpu

# meshes with ragged tiles and a ragged last group of 4 tiles (9x6x5: 18 tiles)
DIMS = [(5, 6, 3), (9, 6, 5), (1, 1, 1), (4, 4, 2)]


def tc_op(dims, k, kind, bc, mass=1.0):
    d = DevOp(*dims, k, "cart", kind, mass, mf.MF_FP64, bc)
    # the default from degree 2; selectable at degree 1
    assert (mf.mf_operator_get_variant(d.op) == mf.MF_VARIANT_TENSOR) == (k >= 2)
    mf.mf_operator_set_variant(d.op, mf.MF_VARIANT_TENSOR)
    return d


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("kind,bc", [(mf.MF_LAPLACE, 0), (mf.MF_HELMHOLTZ, 1), (mf.MF_HELMHOLTZ, 0)])
def test_tensor_apply_matches_oracle(oracle, k, dims, kind, bc):
    d = tc_op(dims, k, kind, bc)
    o = oracle_op(oracle, *dims, k, "cart", 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
    xu = inputs.random_unique(*dims, k, 5)
    y = d.apply(d.native_from_unique(xu))
    err = rel_max(d.canonical_from_native(y), o.scatter(o.apply(xu)))
    assert err <= 1e-12, err
    assert np.isfinite(y.cpu().numpy()).all()  # padding written as 0, no NaN left
    assert mf.mf_device_error() == 0
    d.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_split_apply_is_local_operator(oracle, k):
    dims = (9, 6, 5)
    d = tc_op(dims, k, mf.MF_HELMHOLTZ, 0)
    o = oracle_op(oracle, *dims, k, "cart", 1.0, 0)
    xu = inputs.random_unique(*dims, k, 8)
    ys = d.apply(d.native_from_unique(xu), split=True)
    ref = o.apply_cells(o.scatter(xu), np.arange(o.ncells)).ravel()
    assert rel_max(d.canonical_from_native(ys), ref) <= 1e-12
    d.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_agrees_with_double_float_variants(k):
    d = tc_op((9, 6, 5), k, mf.MF_HELMHOLTZ, 1)
    xn = d.native_from_unique(inputs.random_unique(9, 6, 5, k, 9))
    yt = d.apply(xn)
    yt2 = d.apply(xn)
    torch.cuda.synchronize()
    assert torch.equal(yt, yt2)  # deterministic
    for v in (0, 1, 2):
        mf.mf_operator_set_variant(d.op, v)
        yd = d.apply(xn)
        torch.cuda.synchronize()
        err = float((yd - yt).abs().max() / yd.abs().max())
        assert err <= 1e-12, (v, err)
    mf.mf_operator_set_variant(d.op, mf.MF_VARIANT_TENSOR)
    assert torch.equal(d.apply(xn), yt)
    d.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tensor_apply_commutes_with_powers_of_two(k):
    """Each cell's digits are taken relative to its own largest exponent, so scaling x by
    2^s (no overflow or underflow) scales every output by exactly 2^s."""
    d = tc_op((5, 6, 3), k, mf.MF_LAPLACE, 0)
    xn = d.native_from_unique(inputs.random_unique(5, 6, 3, k, 10))
    y = d.apply(xn)
    for s in (-700, -37, 1, 53, 600):
        ys = d.apply(xn * (2.0 ** s))
        torch.cuda.synchronize()
        assert torch.equal(ys, y * (2.0 ** s)), s
    d.close()


@pytest.mark.parametrize("k", [1, 3])
def test_tensor_apply_values_just_below_powers_of_two(oracle, k):
    """Values within a few ulps below a power of two carry into the top digit (its range is
    [-128, 128]); mixed with random signs and magnitudes they must still match the oracle."""
    dims = (9, 6, 5)
    d = tc_op(dims, k, mf.MF_HELMHOLTZ, 0)
    o = oracle_op(oracle, *dims, k, "cart", 1.0, 0)
    rng = np.random.default_rng(21)
    n = d.n_unique
    e = rng.integers(-3, 4, n).astype(np.float64)
    near = (1.0 - rng.integers(1, 2**20, n) * 2.0**-53) * 2.0**e
    xu = np.where(rng.random(n) < 0.5, near, inputs.random_unique(*dims, k, 22))
    xu *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    y = d.canonical_from_native(d.apply(d.native_from_unique(xu)))
    assert rel_max(y, o.scatter(o.apply(xu))) <= 1e-12
    d.close()


def test_tensor_apply_wide_dynamic_range_and_zeros(oracle):
    """Values spanning ~600 binades: each cell is exact relative to its own largest value, so
    cells of tiny values keep full relative accuracy next to cells of huge ones."""
    dims, k = (9, 6, 5), 3
    d = tc_op(dims, k, mf.MF_HELMHOLTZ, 0)
    o = oracle_op(oracle, *dims, k, "cart", 1.0, 0)
    xu = inputs.random_unique(*dims, k, 11)
    pos = o.node_positions()
    xu = xu * np.where(pos[:, 0] < 0.5, 1e150, 1e-150)
    y = d.canonical_from_native(d.apply(d.native_from_unique(xu)))
    ref = o.scatter(o.apply(xu))
    big = np.abs(ref) > 1e100
    assert rel_max(y[big], ref[big]) <= 1e-12
    # cells entirely in the small region: relative to their own scale
    n3 = (k + 1) ** 3
    yc, rc = y.reshape(-1, n3), ref.reshape(-1, n3)
    small = np.abs(rc).max(axis=1) < 1e-100
    assert small.any()
    assert rel_max(yc[small], rc[small]) <= 1e-12
    z = d.apply(torch.zeros(d.n_native, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert int((z != 0).sum()) == 0
    d.close()


def test_tensor_nonfinite_input_poisons_only_its_cell():
    dims, k = (9, 6, 5), 2
    d = tc_op(dims, k, mf.MF_LAPLACE, 0)
    xn = d.native_from_unique(inputs.random_unique(*dims, k, 12))
    y0 = d.apply(xn, split=True)
    n3 = (k + 1) ** 3
    can = torch.empty(d.n_cw, dtype=torch.float64, device="cuda")
    mf.mf_from_native(d.op, xn.data_ptr(), can.data_ptr())
    cell = 17
    can[cell * n3 + 4] = float("inf")
    xbad = torch.empty_like(xn)
    mf.mf_to_native(d.op, can.data_ptr(), xbad.data_ptr())
    y1 = d.apply(xbad, split=True)
    c0, c1 = d.canonical_from_native(y0).reshape(-1, n3), d.canonical_from_native(y1).reshape(-1, n3)
    assert np.isnan(c1[cell]).all()
    others = np.arange(c0.shape[0]) != cell
    assert np.array_equal(c0[others], c1[others])
    assert mf.mf_device_error() == 0
    d.close()


def test_tensor_variant_refused_where_not_built():
    d = DevOp(5, 6, 3, 4, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)  # degree 4: double-float
    assert mf.mf_operator_get_variant(d.op) == 0
    with pytest.raises(mf.MfError) as e:
        mf.mf_operator_set_variant(d.op, mf.MF_VARIANT_TENSOR)
    assert e.value.code == mf.MF_ERR_UNSUPPORTED
    d.close()
    d = DevOp(5, 6, 3, 2, "curved", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    with pytest.raises(mf.MfError):
        mf.mf_operator_set_variant(d.op, mf.MF_VARIANT_TENSOR)
    d.close()
