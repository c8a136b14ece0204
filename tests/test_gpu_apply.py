"""GPU parity of mf_apply / mf_apply_split / mf_dss / layout helpers against the FP64 oracle.

Tolerances (relative max-norm max|y - y_ref| / max|y_ref|): FP64 1e-12, FP32 1e-5.
Meshes span several 4x4x2 tiles with ragged tails in every direction.
"""
import os

import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._gpu import DevOp, oracle_op, rel_max

pytestmark = pytest.mark.gpu

TOL = {mf.MF_FP64: 1e-12, mf.MF_FP64_DFMA: 1e-12, mf.MF_FP32: 1e-5}

VARIANTS = [
    # geom, kind, bc, precision
    ("cart", mf.MF_LAPLACE, 0, mf.MF_FP64),
    ("curved", mf.MF_HELMHOLTZ, 1, mf.MF_FP64),
    ("shear", mf.MF_LAPLACE, 0, mf.MF_FP64),
    ("stretch", mf.MF_HELMHOLTZ, 0, mf.MF_FP64),
    ("curved", mf.MF_LAPLACE, 0, mf.MF_FP32),
    ("cart", mf.MF_HELMHOLTZ, 1, mf.MF_FP32),
    ("shear", mf.MF_HELMHOLTZ, 1, mf.MF_FP32),
    ("curved", mf.MF_HELMHOLTZ, 1, mf.MF_FP64_DFMA),
    ("cart", mf.MF_LAPLACE, 0, mf.MF_FP64_DFMA),
    ("shear", mf.MF_HELMHOLTZ, 0, mf.MF_FP64_DFMA),
]


def run_parity(oracle, dims, k, geom, kind, bc, prec, seed=3):
    nx, ny, nz = dims
    d = DevOp(nx, ny, nz, k, geom, kind, 1.0, prec, bc)
    o = oracle_op(oracle, nx, ny, nz, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
    xu = inputs.random_unique(nx, ny, nz, k, seed)
    if prec == mf.MF_FP32:
        xu = xu.astype(np.float32).astype(np.float64)  # both sides see the same rounded input
    xn = d.native_from_unique(xu)
    y = d.apply(xn)
    ycan = d.canonical_from_native(y)
    yref = o.scatter(o.apply(xu))
    err = rel_max(ycan, yref)
    # padding lanes are zero, every real copy written (no NaN left from the poisoned buffer)
    yh = y.double().cpu().numpy()
    assert np.isfinite(yh).all()
    d.close()
    return err, ycan, yref


@pytest.mark.parametrize("k", range(1, 9))
@pytest.mark.parametrize("geom,kind,bc,prec", VARIANTS)
def test_apply_parity_ragged(oracle, k, geom, kind, bc, prec):
    dims = (5, 6, 3) if k <= 5 else (5, 2, 3)
    err, _, _ = run_parity(oracle, dims, k, geom, kind, bc, prec)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("bc", [0, 1])
def test_config1_q2_laplace_8cubed(oracle, bc):
    """Q2 Laplace, affine unit cube 8x8x8, FP64, x uniform[-1,1] seed 0: one y = A x."""
    err, _, _ = run_parity(oracle, (8, 8, 8), 2, "cart", mf.MF_LAPLACE, bc, mf.MF_FP64, seed=0)
    assert err <= 1e-12, err


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 2), (3, 1, 1), (4, 4, 2), (9, 1, 5)])
@pytest.mark.parametrize("k", [1, 4])
def test_apply_small_and_degenerate_meshes(oracle, dims, k):
    for geom in ("cart", "curved"):
        err, _, _ = run_parity(oracle, dims, k, geom, mf.MF_HELMHOLTZ, 0, mf.MF_FP64)
        assert err <= 1e-12, (geom, err)


@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("prec", [mf.MF_FP64, mf.MF_FP32])
def test_output_is_consistent_and_deterministic(k, prec):
    """Every copy of a shared node is bitwise equal after the duplicate summation, and two
    applies give bitwise identical results."""
    d = DevOp(5, 6, 3, k, "curved", mf.MF_HELMHOLTZ, 1.0, prec, 0)
    xn = d.native_from_unique(inputs.random_unique(5, 6, 3, k, 11))
    y1 = d.apply(xn)
    y2 = d.apply(xn)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    rebuilt = d.native_from_unique(d.unique_from_native(y1))
    assert torch.equal(rebuilt, y1)
    d.close()


@pytest.mark.parametrize("k", [2, 5])
def test_split_apply_is_local_operator(oracle, k):
    """mf_apply_split returns A_K x_K per cell (Eq. (split_operator)); mf_dss of it equals mf_apply."""
    dims = (5, 6, 3)
    d = DevOp(*dims, k, "curved", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    o = oracle_op(oracle, *dims, k, "curved", 0.0, 0)
    xu = inputs.random_unique(*dims, k, 5)
    xn = d.native_from_unique(xu)
    ys = d.apply(xn, split=True)
    ref = o.apply_cells(o.scatter(xu), np.arange(o.ncells)).ravel()
    assert rel_max(d.canonical_from_native(ys), ref) <= 1e-12
    mf.mf_dss(d.op, ys.data_ptr())
    assert torch.equal(ys, d.apply(xn))
    d.close()


def test_layout_round_trip():
    d = DevOp(5, 6, 3, 3, "cart")
    can = torch.arange(d.n_cw, dtype=torch.float64, device="cuda")
    nat = torch.full((d.n_native,), -1.0, dtype=torch.float64, device="cuda")
    mf.mf_to_native(d.op, can.data_ptr(), nat.data_ptr())
    back = torch.zeros(d.n_cw, dtype=torch.float64, device="cuda")
    mf.mf_from_native(d.op, nat.data_ptr(), back.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(back, can)
    # native holds every canonical value exactly once; padding lanes are zero
    npad = d.n_native - d.n_cw
    assert int((nat == 0).sum()) == npad + 1
    assert torch.equal(torch.sort(nat).values[npad:], can)
    d.close()


@pytest.mark.parametrize("prec,bc", [(mf.MF_FP64, 0), (mf.MF_FP32, 0), (mf.MF_FP64, 1)])
@pytest.mark.parametrize("k,dims", [(1, (5, 6, 3)), (3, (5, 6, 3)), (6, (5, 2, 3))])
def test_make_consistent_is_average_of_copies(oracle, prec, bc, k, dims):
    """mf_make_consistent against the oracle's assembly G^T divided by the multiplicity
    (assemble(1)), gathered back to every copy (Sec. 4, Eqs. (shadow_gather),
    (shadow_assembly)); no Dirichlet mask.  All copies bitwise equal; a consistent vector
    is left unchanged."""
    d = DevOp(*dims, k, "cart", mf.MF_LAPLACE, 1.0, prec, bc)
    o = oracle_op(oracle, *dims, k, "cart", 0.0, bc)
    rng = np.random.default_rng(7)
    ycw = rng.uniform(-1.0, 1.0, d.n_cw)  # independent copies: not consistent
    if prec == mf.MF_FP32:
        ycw = ycw.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == mf.MF_FP32 else torch.float64
    can = torch.as_tensor(ycw, dtype=dt, device="cuda")
    nat = torch.empty(d.n_native, dtype=dt, device="cuda")
    mf.mf_to_native(d.op, can.data_ptr(), nat.data_ptr())
    mf.mf_make_consistent(d.op, nat.data_ptr())
    got = d.canonical_from_native(nat)
    ref = o.scatter(o.assemble(ycw) / o.assemble(np.ones(d.n_cw)))
    assert rel_max(got, ref) <= (1e-6 if prec == mf.MF_FP32 else 1e-15)
    # every copy of a node equal: gathering one copy and scattering it back changes nothing
    back = d.native_from_unique(d.unique_from_native(nat))
    assert torch.equal(back, nat)
    # idempotent (a projection onto consistent vectors)
    again = nat.clone()
    mf.mf_make_consistent(d.op, again.data_ptr())
    assert torch.equal(again, nat)
    d.close()


@pytest.mark.parametrize("prec", [mf.MF_FP64, mf.MF_FP32])
def test_dot_products(oracle, prec):
    """Assembled dot over unique nodes (1/multiplicity weights) and the Lemma 1 pairing of a
    split dual with a consistent primal."""
    dims, k = (5, 6, 3), 3
    d = DevOp(*dims, k, "curved", mf.MF_HELMHOLTZ, 1.0, prec, 0)
    o = oracle_op(oracle, *dims, k, "curved", 1.0, 0)
    a = inputs.random_unique(*dims, k, 21)
    b = inputs.random_unique(*dims, k, 22)
    if prec == mf.MF_FP32:
        a = a.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    an, bn = d.native_from_unique(a), d.native_from_unique(b)
    got = d.dot(an, bn)
    assert abs(got - a @ b) <= 1e-13 * np.abs(a * b).sum()
    ys = d.apply(an, split=True)
    pair = d.dot(ys, bn, split=1)
    ref = o.apply(a) @ b
    assert abs(pair - ref) <= TOL[prec] * np.abs(o.apply(a)).max() * np.abs(b).sum()
    d.close()


@pytest.mark.parametrize("scale", [1e-200, 1e-25, 1.0, 1e25, 1e200])
def test_dot_keeps_the_double_range(scale):
    """The FP64 dot accumulates on the FP32 pipe for operands within [2^-60, 2^60] and in FP64
    outside; over the whole double range (both paths in one dot: half of b sits 30 decades
    lower) it stays within 1e-13 of the exactly rounded sum."""
    import math
    dims, k = (5, 4, 3), 2
    d = DevOp(*dims, k, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    a = inputs.random_unique(*dims, k, 31) * scale
    b = inputs.random_unique(*dims, k, 32)
    b[::2] *= 1e-30
    got = d.dot(d.native_from_unique(a), d.native_from_unique(b))
    ref = math.fsum(a * b)
    assert abs(got - ref) <= 1e-13 * np.abs(a * b).sum(), (got, ref)
    d.close()


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("prec", [mf.MF_FP64, mf.MF_FP32, mf.MF_FP64_DFMA])
def test_full_size_curved_64cubed_sampled(oracle, k, prec):
    """Q3/Q4 Laplace on the curved 64^3 mesh, seed 1, FP64 and FP32: sampled global nodes are
    compared with the oracle's sum of the local results of the cells sharing them."""
    N = 64
    d = DevOp(N, N, N, k, "curved", mf.MF_LAPLACE, 1.0, prec, 0)
    xu = inputs.random_unique(N, N, N, k, 1)
    if prec == mf.MF_FP32:
        xu = xu.astype(np.float32).astype(np.float64)
    y = d.unique_from_native(d.apply(d.native_from_unique(xu)))
    o = oracle_op(oracle, N, N, N, k, "curved", 0.0, 0)
    check_sampled(o, xu, y, TOL[prec], seed=k)
    d.close()


def check_sampled(o, xu, y, tol, seed, nsample=120):
    k, n = o.k, o.k + 1
    NX, NY = o.nx * k + 1, o.ny * k + 1
    rng = np.random.default_rng(seed)
    nodes = rng.integers(0, o.n_unique, nsample)
    nodes[:4] = [0, o.n_unique - 1, (o.n_unique // 2), NX * NY + NX + 1]
    cells, locs = [], []
    for g in nodes:
        I, J, L = g % NX, (g // NX) % NY, g // (NX * NY)
        lst = []
        for cx, i in _copies(I, o.nx, k):
            for cy, j in _copies(J, o.ny, k):
                for cz, l in _copies(L, o.nz, k):
                    lst.append(((cz * o.ny + cy) * o.nx + cx, i + n * (j + n * l)))
        locs.append(lst)
        cells += [c for c, _ in lst]
    ucells = np.unique(np.array(cells, dtype=np.int64))
    # canonical cell-wise x only for the needed cells
    xcw = np.zeros((o.ncells, n ** 3))
    dofs = _cell_dofs_subset(o, ucells)
    xcw[ucells] = xu[dofs]
    yl = o.apply_cells(xcw.ravel(), ucells)
    pos = {c: m for m, c in enumerate(ucells)}
    ref = np.array([sum(yl[pos[c], l] for c, l in lst) for lst in locs])
    got = y[nodes]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale, (np.abs(got - ref).max() / scale)


def _copies(I, nc, k):
    c = I // k
    if I % k == 0:
        out = []
        if c > 0:
            out.append((c - 1, k))
        if c < nc:
            out.append((c, 0))
        return out
    return [(c, I - c * k)]


def _cell_dofs_subset(o, cells):
    k, n = o.k, o.k + 1
    NX, NY = o.nx * k + 1, o.ny * k + 1
    cx = cells % o.nx
    cy = (cells // o.nx) % o.ny
    cz = cells // (o.nx * o.ny)
    i = np.arange(n)
    I = cx[:, None, None, None] * k + i[None, None, None, :]
    J = cy[:, None, None, None] * k + i[None, None, :, None]
    L = cz[:, None, None, None] * k + i[None, :, None, None]
    return (I + NX * (J + NY * L)).reshape(len(cells), -1)


@pytest.mark.parametrize("k,N", [(1, 184), (2, 123), (3, 92), (4, 74), (5, 61), (6, 53), (7, 46), (8, 41)])
@pytest.mark.parametrize("prec", [mf.MF_FP64, mf.MF_FP64_DFMA])
def test_full_size_helmholtz_sweep_sampled(oracle, k, N, prec):
    """Degree sweep: Helmholtz (M + K) on the affine unit cube with ~50M cell-wise DoFs,
    FP64, seed 2 -- sampled against the oracle."""
    d = DevOp(N, N, N, k, "cart", mf.MF_HELMHOLTZ, 1.0, prec, 0)
    xu = inputs.random_unique(N, N, N, k, 2)
    y = d.unique_from_native(d.apply(d.native_from_unique(xu)))
    o = oracle_op(oracle, N, N, N, k, "cart", 1.0, 0)
    check_sampled(o, xu, y, 1e-12, seed=k, nsample=60)
    d.close()


@pytest.mark.parametrize("k,geom,prec", [(2, "cart", mf.MF_FP64), (4, "curved", mf.MF_FP64), (5, "curved", mf.MF_FP32),
                                         (8, "shear", mf.MF_FP64), (3, "curved", mf.MF_FP64_DFMA)])
def test_launch_variants_agree_bitwise_and_autotune(k, geom, prec):
    """Both launch configurations run the same per-thread arithmetic: bitwise equal output.
    The autotuner picks one of them and leaves the result unchanged."""
    d = DevOp(5, 6, 3, k, geom, mf.MF_HELMHOLTZ, 1.0, prec, 0)
    xn = d.native_from_unique(inputs.random_unique(5, 6, 3, k, 13))
    mf.mf_operator_set_variant(d.op, 0)
    y0 = d.apply(xn)
    variants = (1, 2, mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY) if prec == mf.MF_FP64 else (1, 2)
    for v in variants:
        mf.mf_operator_set_variant(d.op, v)
        y1 = d.apply(xn)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1), v
    if prec != mf.MF_FP64:  # variants 4 and 5 are built for the double-float view only
        for v in (mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY):
            with pytest.raises(mf.MfError) as e:
                mf.mf_operator_set_variant(d.op, v)
            assert e.value.code == mf.MF_ERR_UNSUPPORTED
    scratch = torch.empty_like(xn)
    v = mf.mf_operator_autotune(d.op, xn.data_ptr(), scratch.data_ptr(), 2)
    if v == mf.MF_VARIANT_TENSOR:  # the tensor-core apply rounds differently (same accuracy)
        assert geom == "cart" and prec == mf.MF_FP64 and k <= 3
        y3 = d.apply(xn)
        torch.cuda.synchronize()
        assert float((y3 - y0).abs().max() / y0.abs().max()) <= 1e-12
    else:
        assert v in variants or v == 0
        assert torch.equal(d.apply(xn), y0)
    d.close()


@pytest.mark.parametrize("prec,dims,k,bc", [(mf.MF_FP64, (7, 6, 5), 3, 0), (mf.MF_FP64, (5, 9, 4), 5, 1),
                                             (mf.MF_FP32, (6, 5, 7), 4, 1)])
def test_atomic_dss_ablation_matches_sweep_dss(prec, dims, k, bc):
    """The atomic duplicate summation (ablation entry) gives the sweep's sums up to the order
    of the additions, and a consistent vector."""
    d = DevOp(*dims, k, "curved", mf.MF_LAPLACE, 1.0, prec, bc)
    x = d.native_from_unique(inputs.random_unique(*dims, k, 41))
    ys = d.apply(x, split=True)
    y_sweep = ys.clone()
    mf.mf_dss(d.op, y_sweep.data_ptr())
    y_atomic = ys.clone()
    sc = torch.empty(max(mf.mf_dss_atomic_workspace_bytes(d.op), 256), dtype=torch.uint8, device="cuda")
    mf.mf_dss_atomic(d.op, y_atomic.data_ptr(), sc.data_ptr(), sc.numel())
    torch.cuda.synchronize()
    a, b = y_atomic.double().cpu().numpy(), y_sweep.double().cpu().numpy()
    tol = 1e-6 if prec == mf.MF_FP32 else 1e-14
    assert np.abs(a - b).max() <= tol * np.abs(b).max()
    u = torch.empty(d.n_unique, dtype=d.dtype, device="cuda")
    mf.mf_gather_unique(d.op, y_atomic.data_ptr(), u.data_ptr())
    back = torch.empty_like(y_atomic)
    mf.mf_scatter_unique(d.op, u.data_ptr(), back.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(back, y_atomic)
    d.close()


@pytest.mark.parametrize("variant", [0, 1, mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY])
@pytest.mark.parametrize("geom,kind,prec,k,dims", [
    ("curved", mf.MF_LAPLACE, mf.MF_FP64, 4, (5, 6, 3)),
    ("curved", mf.MF_HELMHOLTZ, mf.MF_FP64, 1, (9, 5, 3)),
    ("curved", mf.MF_LAPLACE, mf.MF_FP64, 8, (5, 2, 3)),
    ("curved", mf.MF_HELMHOLTZ, mf.MF_FP64_DFMA, 2, (5, 6, 3)),
    ("curved", mf.MF_LAPLACE, mf.MF_MIXED, 3, (5, 6, 3)),
    ("curved", mf.MF_LAPLACE, mf.MF_FP32, 3, (5, 6, 3)),
    ("curved", mf.MF_HELMHOLTZ, mf.MF_FP32, 8, (5, 2, 3)),
    ("cart", mf.MF_HELMHOLTZ, mf.MF_FP64, 5, (5, 6, 3)),
    ("shear", mf.MF_LAPLACE, mf.MF_FP32, 6, (5, 2, 3)),
])
def test_stream_twin_copies_x(geom, kind, prec, k, dims, variant):
    """The stream twin (the apply's accesses without its arithmetic) writes every native
    element, padding lanes included, as a bit-copy of x, for every view and launch variant."""
    if variant in (mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY) and prec != mf.MF_FP64:
        pytest.skip("variants 4 and 5 are built for the double-float view only")
    d = DevOp(*dims, k, geom, kind, 1.0, prec, 0)
    mf.mf_operator_set_variant(d.op, variant)
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn(d.n_native, dtype=d.dtype, device="cuda", generator=g)
    y = torch.full_like(x, float("nan"))
    mf.mf_apply_stream_twin(d.op, x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    ib = torch.int64 if d.dtype == torch.float64 else torch.int32
    assert torch.equal(y.view(ib), x.view(ib))
    with pytest.raises(mf.MfError):
        mf.mf_apply_stream_twin(d.op, x.data_ptr(), x.data_ptr())
    d.close()


def test_autotune_choice_persists_in_json_file(tmp_path):
    """The autotuner writes its choice to the JSON cache keyed by the GPU's name, and a fresh
    process takes a stored choice from the file instead of timing (a planted entry wins)."""
    import json
    import subprocess
    import sys

    cache = tmp_path / "autotune.json"
    code = (
        "import sys, torch; sys.path.insert(0, %r)\n"
        "import paper_2609_04534_gb300 as mf\n"
        "from paper_2609_04534_gb300 import inputs\n"
        "from tests._gpu import DevOp\n"
        "d = DevOp(5, 6, 3, 4, 'curved', mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)\n"
        "x = d.native_from_unique(inputs.random_unique(5, 6, 3, 4, 3)); y = torch.empty_like(x)\n"
        "print(mf.mf_operator_autotune(d.op, x.data_ptr(), y.data_ptr(), 2))\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),)
    env = dict(os.environ, MF_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    v = int(r.stdout.strip().splitlines()[-1])
    entries = json.loads(cache.read_text())
    keys = [k for k in entries if "|n=5|path=2|" in k]
    assert len(keys) == 1 and entries[keys[0]] == v and torch.cuda.get_device_name(0) in keys[0]
    planted = (v + 1) % 3
    entries[keys[0]] = planted
    cache.write_text(json.dumps(entries))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert int(r.stdout.strip().splitlines()[-1]) == planted


@pytest.mark.parametrize("geom,prec,kind", [("cart", mf.MF_FP64, mf.MF_LAPLACE), ("curved", mf.MF_FP64, mf.MF_HELMHOLTZ),
                                            ("shear", mf.MF_FP32, mf.MF_LAPLACE), ("cart", mf.MF_FP32, mf.MF_HELMHOLTZ),
                                            ("curved", mf.MF_FP32, mf.MF_HELMHOLTZ)])
def test_block_size_sweep_matches_split_apply(oracle, geom, prec, kind):
    """The block-size sweep (B = 4, 8, 16, 32 cells per CTA, degree 3) computes each cell with
    the arithmetic of launch variant 0: bitwise the same split result, on a ragged mesh whose
    tiles are partly outside it; the FP64 result also matches the oracle's local apply."""
    k, dims = 3, (9, 6, 5)
    d = DevOp(*dims, k, geom, kind, 1.0, prec, 0)
    xu = inputs.random_unique(*dims, k, 21)
    xn = d.native_from_unique(xu)
    mf.mf_operator_set_variant(d.op, 0)
    y0 = d.apply(xn, split=True)
    for b in (4, 8, 16, 32):
        y = torch.full_like(y0, float("nan"))
        mf.mf_apply_split_block(d.op, b, xn.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(y, y0), b
    if prec == mf.MF_FP64:
        o = oracle_op(oracle, *dims, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, 0)
        ref = o.apply_cells(o.scatter(xu), np.arange(o.ncells)).ravel()
        got = d.canonical_from_native(y0)
        assert rel_max(got, ref) <= 1e-12
    d.close()


@pytest.mark.parametrize("k", [1, 2, 4, 5, 6, 7, 8])
def test_block_size_sweep_cartesian_every_degree(oracle, k):
    """The Cartesian double-float apply with B cells per CTA, at every degree and every B that
    makes a CTA of 32..1024 threads: bitwise launch variant 0's split result."""
    dims = (9, 6, 5)
    d = DevOp(*dims, k, "cart", mf.MF_HELMHOLTZ, 1.0, mf.MF_FP64, 0)
    xn = d.native_from_unique(inputs.random_unique(*dims, k, 22))
    mf.mf_operator_set_variant(d.op, 0)
    y0 = d.apply(xn, split=True)
    n = k + 1
    for b in (4, 8, 16, 32):
        if not 32 <= n * n * b <= 1024:
            continue
        y = torch.full_like(y0, float("nan"))
        mf.mf_apply_split_block(d.op, b, xn.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(y, y0), b
    d.close()


def test_block_size_sweep_refusals():
    """Combinations that are not built -- the curved path and FP32 away from degree 3, CTAs
    outside 32..1024 threads, the native-FP64 (DFMA) view of MF_FP64_DFMA and MF_MIXED -- are
    refused before any launch."""
    for k, geom, prec, b in ((2, "curved", mf.MF_FP64, 8), (5, "cart", mf.MF_FP32, 8), (1, "cart", mf.MF_FP64, 4),
                             (7, "cart", mf.MF_FP64, 32)):
        d = DevOp(4, 4, 4, k, geom, mf.MF_LAPLACE, 1.0, prec, 0)
        dt = torch.float32 if prec == mf.MF_FP32 else torch.float64
        x = torch.zeros(d.n_native, dtype=dt, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(mf.MfError) as e:
            mf.mf_apply_split_block(d.op, b, x.data_ptr(), y.data_ptr())
        assert e.value.code == mf.MF_ERR_UNSUPPORTED, (k, geom, prec, b)
        d.close()
    for prec in (mf.MF_FP64_DFMA, mf.MF_MIXED):
        d = DevOp(4, 4, 4, 3, "cart", mf.MF_LAPLACE, 1.0, prec, 0)
        x = torch.zeros(d.n_native, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(mf.MfError) as e:
            mf.mf_apply_split_block(d.op, 8, x.data_ptr(), y.data_ptr())
        assert e.value.code == mf.MF_ERR_UNSUPPORTED
        d.close()
