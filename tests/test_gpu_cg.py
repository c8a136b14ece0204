"""GPU CG and mixed-precision defect correction against the oracle's textbook CG."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._gpu import DevOp, oracle_op, rel_max

pytestmark = pytest.mark.gpu


def solve(d, b, rtol, maxit, mixed, hist_cap=0, cg_form=0, mixed_restart=0):
    x = torch.zeros(d.n_native, dtype=d.dtype, device="cuda")
    ws = torch.empty(mf.mf_cg_workspace_bytes(d.op, mixed), dtype=torch.uint8, device="cuda")
    hist = np.zeros(max(hist_cap, 1))
    if hist_cap:
        mf.mf_cg_record_history(hist.ctypes.data, hist_cap)
    try:
        st = mf.mf_cg_solve(d.op, b.data_ptr(), x.data_ptr(), rtol, maxit, mixed, ws.data_ptr(), ws.numel(),
                            allow_not_converged=True, cg_form=cg_form, mixed_restart=mixed_restart)
    finally:
        mf.mf_cg_record_history(None, 0)
    return x, st, hist


@pytest.mark.parametrize("cg_form", [mf.MF_CG_SPLIT_DUAL, mf.MF_CG_ASSEMBLED])
def test_config1_50_cg_iterations(oracle, cg_form):
    """Q2 Laplace 8^3, Dirichlet, b = A x_true with x_true the seed-0 random vector masked at
    the boundary; 50 CG iterations from 0.  Per-iteration relative residuals and x_50 agree
    with the oracle within 1e-10, for both forms of the iteration."""
    N, k = 8, 2
    d = DevOp(N, N, N, k, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 1)
    o = oracle_op(oracle, N, N, N, k, "cart", 0.0, 1)
    xt = inputs.random_unique(N, N, N, k, 0)
    xt[o.boundary_mask()] = 0.0
    b_ref = o.apply(xt)
    x_ref, h_ref = o.cg(b_ref, maxit=50, rtol=0.0)
    b = d.apply(d.native_from_unique(xt))
    x, st, h = solve(d, b, 0.0, 50, 0, hist_cap=64, cg_form=cg_form)
    assert st["iterations"] == 50
    np.testing.assert_allclose(h[:51], h_ref, rtol=1e-10, atol=0)
    assert rel_max(d.unique_from_native(x), x_ref) <= 1e-10
    d.close()


@pytest.mark.parametrize("geom,k", [("curved", 2), ("cart", 3)])
def test_fp64_cg_converges_to_oracle_solution(oracle, geom, k):
    N = 5
    d = DevOp(N, N, N, k, geom, mf.MF_LAPLACE, 1.0, mf.MF_FP64, 1)
    o = oracle_op(oracle, N, N, N, k, geom, 0.0, 1)
    bu = inputs.random_unique(N, N, N, k, 7)
    x, st, _ = solve(d, d.native_from_unique(bu), 1e-10, 5000, 0)
    assert st["code"] == mf.MF_OK and st["rel_residual"] <= 1e-10
    xg = d.unique_from_native(x)
    bm = np.where(o.boundary_mask(), 0.0, bu)
    res = np.linalg.norm(bm - o.apply(xg)) / np.linalg.norm(bm)
    assert res <= 2e-10
    d.close()


@pytest.mark.parametrize("geom,kind,cg_form,restart", [
    ("curved", mf.MF_LAPLACE, 0, 0), ("shear", mf.MF_HELMHOLTZ, 0, 0), ("curved", mf.MF_LAPLACE, 0, 1),
    ("shear", mf.MF_HELMHOLTZ, 0, 1), ("curved", mf.MF_LAPLACE, mf.MF_CG_ASSEMBLED, 0),
    ("shear", mf.MF_LAPLACE, mf.MF_CG_SPLIT_DUAL_FUSED, 0)])
def test_mixed_precision_defect_correction(oracle, geom, kind, cg_form, restart):
    """FP32 inner CG inside FP64 defect correction -- continued with reliable updates
    (restart = 0) or restarted at every defect-correction step -- reaches the FP64 tolerance
    1e-10 (true residual checked by the oracle) and matches the FP64 solve, for every form of
    the inner iteration."""
    N, k = 6, 3
    d = DevOp(N, N, N, k, geom, kind, 1.0, mf.MF_MIXED, 1)
    o = oracle_op(oracle, N, N, N, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, 1)
    bu = inputs.random_unique(N, N, N, k, 9)
    b = d.native_from_unique(bu)
    x, st, _ = solve(d, b, 1e-10, 20000, 1, cg_form=cg_form, mixed_restart=restart)
    assert st["code"] == mf.MF_OK, st
    assert st["outer_iterations"] >= 2
    xg = d.unique_from_native(x)
    bm = np.where(o.boundary_mask(), 0.0, bu)
    res = np.linalg.norm(bm - o.apply(xg)) / np.linalg.norm(bm)
    assert res <= 2e-10, res
    x64, st64, _ = solve(d, b, 1e-10, 20000, 0)
    assert st64["code"] == mf.MF_OK
    assert rel_max(xg, d.unique_from_native(x64)) <= 1e-7
    d.close()


@pytest.mark.parametrize("geom,k", [("curved", 4), ("cart", 2)])
def test_reliable_updates_keep_the_krylov_space(oracle, geom, k):
    """With reliable updates the inner CG continues across defect-correction steps: on a
    problem that needs several outer steps it takes fewer inner iterations in total than the
    restarted inner CG, and both reach 1e-10 with the true residual checked by the oracle."""
    N = 10
    d = DevOp(N, N, N, k, geom, mf.MF_LAPLACE, 1.0, mf.MF_MIXED, 1)
    o = oracle_op(oracle, N, N, N, k, geom, 0.0, 1)
    bu = inputs.random_unique(N, N, N, k, 4)
    b = d.native_from_unique(bu)
    bm = np.where(o.boundary_mask(), 0.0, bu)
    its = {}
    for restart in (0, 1):
        x, st, _ = solve(d, b, 1e-10, 20000, 1, mixed_restart=restart)
        assert st["code"] == mf.MF_OK, st
        res = np.linalg.norm(bm - o.apply(d.unique_from_native(x))) / np.linalg.norm(bm)
        assert res <= 2e-10, (restart, res)
        its[restart] = (st["iterations"], st["outer_iterations"])
    assert its[1][1] >= 3, its
    assert its[0][0] < its[1][0], its
    d.close()


def test_breakdown_is_reported():
    """An all-zero operator (Laplace on a 1x1x1 Dirichlet mesh of degree 1 has no free node)
    gives x = 0 immediately; a non-finite right-hand side reports a breakdown, not a hang."""
    d = DevOp(1, 1, 1, 1, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 1)
    b = torch.zeros(d.n_native, dtype=torch.float64, device="cuda")
    x, st, _ = solve(d, b, 1e-10, 10, 0)
    assert st["code"] == mf.MF_OK and st["iterations"] == 0
    d.close()
    d = DevOp(3, 3, 3, 2, "cart", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 0)
    b = d.native_from_unique(inputs.random_unique(3, 3, 3, 2, 1))
    b[5] = float("inf")
    with pytest.raises(mf.MfError) as e:
        solve(d, b, 1e-10, 10, 0)
    assert e.value.code == mf.MF_ERR_BREAKDOWN
    d.close()


def consistent(d, x):
    """All copies of every node bitwise equal (and padding zero): x == G G^T-free round trip."""
    u = torch.empty(d.n_unique, dtype=d.dtype, device="cuda")
    mf.mf_gather_unique(d.op, x.data_ptr(), u.data_ptr())
    xs = torch.empty_like(x)
    mf.mf_scatter_unique(d.op, u.data_ptr(), xs.data_ptr())
    torch.cuda.synchronize()
    return bool(torch.equal(xs, x))


@pytest.mark.parametrize("dims,k,geom,kind,prec,bc", [
    ((7, 6, 5), 3, "curved", mf.MF_LAPLACE, mf.MF_FP64, 1),
    ((9, 5, 3), 2, "shear", mf.MF_HELMHOLTZ, mf.MF_FP64, 0),
    ((5, 9, 4), 4, "cart", mf.MF_LAPLACE, mf.MF_FP64, 1),
    ((6, 7, 5), 5, "curved", mf.MF_HELMHOLTZ, mf.MF_FP64_DFMA, 0),
    ((4, 4, 2), 1, "cart", mf.MF_HELMHOLTZ, mf.MF_FP64, 0),
    ((5, 3, 7), 8, "stretch", mf.MF_LAPLACE, mf.MF_FP64, 1),
    ((7, 6, 5), 3, "curved", mf.MF_LAPLACE, mf.MF_FP32, 1),
    ((9, 5, 3), 6, "cart", mf.MF_HELMHOLTZ, mf.MF_FP32, 0),
])
def test_split_dual_matches_assembled_iteration(oracle, dims, k, geom, kind, prec, bc):
    """The split-dual iteration (fused apply with <p, A_K p> over all copies, duplicate
    summation folded into the update of r) against the assembled iteration (apply, duplicate
    summation, vector kernels), on ragged meshes whose cells cross tile boundaries in every
    direction: the residual histories agree to rounding, the iterates stay consistent
    bitwise, and the split-dual solution satisfies the oracle's equations."""
    nx, ny, nz = dims
    d = DevOp(nx, ny, nz, k, geom, kind, 1.0, prec, bc)
    # both forms on the same apply arithmetic (the assembled form would otherwise take the
    # tensor-core apply of a Cartesian FP64 operator, which rounds differently; CG amplifies
    # such 2^-48 differences to ~1e-8 after 25 iterations): this compares the iterations
    tensor = mf.mf_operator_get_variant(d.op) == mf.MF_VARIANT_TENSOR
    if tensor:
        mf.mf_operator_set_variant(d.op, 0)
    bu = inputs.random_unique(nx, ny, nz, k, 11)
    b = d.native_from_unique(bu)
    its = 25
    xa, sta, ha = solve(d, b, 0.0, its, 0, hist_cap=its + 2, cg_form=mf.MF_CG_ASSEMBLED)
    assert sta["iterations"] == its and consistent(d, xa)
    tol = 1e-3 if prec == mf.MF_FP32 else 1e-9
    for form in (mf.MF_CG_SPLIT_DUAL, mf.MF_CG_SPLIT_DUAL_FUSED):
        xs, sts, hs = solve(d, b, 0.0, its, 0, hist_cap=its + 2, cg_form=form)
        assert sts["iterations"] == its
        np.testing.assert_allclose(hs[:its + 1], ha[:its + 1], rtol=tol, atol=0)
        assert consistent(d, xs)
        assert rel_max(d.unique_from_native(xs), d.unique_from_native(xa)) <= tol
    if prec != mf.MF_FP32:
        o = oracle_op(oracle, nx, ny, nz, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
        bm = np.where(o.boundary_mask(), 0.0, bu) if bc else bu
        forms = [mf.MF_CG_DEFAULT]
        if tensor:  # the assembled iteration on the tensor-core apply solves the same equations
            mf.mf_operator_set_variant(d.op, mf.MF_VARIANT_TENSOR)
            forms.append(mf.MF_CG_ASSEMBLED)
        for form in forms:
            x1, st1, _ = solve(d, b, 1e-11, 20000, 0, cg_form=form)
            assert st1["code"] == mf.MF_OK
            res = np.linalg.norm(bm - o.apply(d.unique_from_native(x1))) / np.linalg.norm(bm)
            assert res <= 2e-11, (form, res)
    d.close()


@pytest.mark.parametrize("scale", [1e-200, 3e-30, 7e25, 1e200])
def test_fp64_cg_across_the_double_range(scale):
    """The FP64 solver's double-float iteration scales b by a power of two near 1/||b|| (so its
    float exponents stay in range) and scales x back: right-hand sides anywhere in the double
    range give the same relative residual history and the correspondingly scaled solution."""
    N, k = 5, 3
    d = DevOp(N, N, N, k, "curved", mf.MF_LAPLACE, 1.0, mf.MF_FP64, 1)
    bu = inputs.random_unique(N, N, N, k, 13)
    x0, st0, h0 = solve(d, d.native_from_unique(bu), 1e-10, 5000, 0, hist_cap=4000)
    x1, st1, h1 = solve(d, d.native_from_unique(bu * scale), 1e-10, 5000, 0, hist_cap=4000)
    assert st0["code"] == st1["code"] == mf.MF_OK
    assert abs(st0["iterations"] - st1["iterations"]) <= 2
    m = min(st0["iterations"], st1["iterations"]) + 1
    np.testing.assert_allclose(h1[:m], h0[:m], rtol=1e-8, atol=0)
    u0, u1 = d.unique_from_native(x0), d.unique_from_native(x1)
    assert np.isfinite(u1).all()
    assert rel_max(u1 / scale, u0) <= 1e-8
    d.close()


@pytest.mark.parametrize("dims,k,geom,kind,bc", [
    ((3, 4, 2), 2, "cart", mf.MF_LAPLACE, 1),
    ((3, 2, 3), 3, "shear", mf.MF_HELMHOLTZ, 0),
    ((2, 3, 2), 4, "curved", mf.MF_LAPLACE, 1),
    ((5, 2, 3), 2, "curved", mf.MF_HELMHOLTZ, 0),
    ((2, 2, 2), 6, "stretch", mf.MF_LAPLACE, 0),
])
def test_diagonal_matches_assembled_matrix(oracle, dims, k, geom, kind, bc):
    """mf_diagonal (FP32, for Jacobi) equals the diagonal of the brute-force assembled sparse
    matrix of the oracle's element matrices (P A P for Dirichlet), within FP32 rounding."""
    from tests._fem_ref import assemble_csr

    d = DevOp(*dims, k, geom, kind, 1.0, mf.MF_FP64, bc)
    o = oracle_op(oracle, *dims, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
    ref = assemble_csr(o, dirichlet=bool(bc)).diagonal()
    dg = torch.empty(d.n_native, dtype=torch.float32, device="cuda")
    sc = torch.empty(max(mf.mf_diagonal_workspace_bytes(d.op), 256), dtype=torch.uint8, device="cuda")
    mf.mf_diagonal(d.op, dg.data_ptr(), sc.data_ptr(), sc.numel())
    dg64 = dg.double()  # the layout helpers use the operator's precision (FP64 here)
    u = torch.empty(d.n_unique, dtype=torch.float64, device="cuda")
    mf.mf_gather_unique(d.op, dg64.data_ptr(), u.data_ptr())
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    d.close()


@pytest.mark.parametrize("geom,k,prec,mixed", [("curved", 3, mf.MF_FP64, 0), ("cart", 4, mf.MF_FP64, 0),
                                               ("curved", 4, mf.MF_MIXED, 1), ("stretch", 2, mf.MF_FP64, 0)])
def test_jacobi_pcg_converges_with_fewer_iterations(oracle, geom, k, prec, mixed):
    """Jacobi-preconditioned CG (split-dual) reaches 1e-10 (true residual checked by the oracle)
    in fewer iterations than plain CG, on meshes where the diagonal varies (stretched cells,
    curved map, high degree).  The mixed solve compares like with like: the preconditioned
    inner CG is restarted at every defect-correction step, so the plain one is too."""
    N = 6
    d = DevOp(N, N + 1, N - 1, k, geom, mf.MF_LAPLACE, 1.0, prec, 1)
    o = oracle_op(oracle, N, N + 1, N - 1, k, geom, 0.0, 1)
    bu = inputs.random_unique(N, N + 1, N - 1, k, 17)
    b = d.native_from_unique(bu)
    x0, st0, _ = solve(d, b, 1e-10, 20000, mixed, mixed_restart=mixed)
    x1 = torch.zeros(d.n_native, dtype=d.dtype, device="cuda")
    ws = torch.empty(mf.mf_cg_workspace_bytes(d.op, mixed), dtype=torch.uint8, device="cuda")
    st1 = mf.mf_cg_solve(d.op, b.data_ptr(), x1.data_ptr(), 1e-10, 20000, mixed, ws.data_ptr(), ws.numel(),
                         precond=mf.MF_PRECOND_JACOBI)
    assert st0["code"] == st1["code"] == mf.MF_OK
    assert st1["iterations"] < st0["iterations"], (st1["iterations"], st0["iterations"])
    xg = d.unique_from_native(x1)
    bm = np.where(o.boundary_mask(), 0.0, bu)
    res = np.linalg.norm(bm - o.apply(xg)) / np.linalg.norm(bm)
    assert res <= 2e-10, res
    assert rel_max(xg, d.unique_from_native(x0)) <= 1e-7
    d.close()


@pytest.mark.parametrize("geom,k,prec", [("curved", 4, mf.MF_FP64), ("cart", 3, mf.MF_FP64), ("curved", 2, mf.MF_FP32)])
def test_cg_solve_host_matches_device_solve(geom, k, prec):
    """mf_cg_solve_host (canonical host b in, canonical host x out) runs the same solve as
    mf_cg_solve on native device vectors: bitwise equal solution and statistics."""
    dims = (5, 6, 3)
    d = DevOp(*dims, k, geom, mf.MF_LAPLACE, 1.0, prec, 1)
    bu = inputs.random_unique(*dims, k, 17)
    b = d.native_from_unique(bu)
    x, st, _ = solve(d, b, 1e-9, 2000, 0)
    xc = d.canonical_from_native(x)
    bh = torch.empty(d.n_cw, dtype=d.dtype, pin_memory=True)
    bh.copy_(torch.as_tensor(d.canonical_from_native(b), dtype=d.dtype))
    xh = torch.full((d.n_cw,), float("nan"), dtype=d.dtype).pin_memory()
    ws = torch.empty(mf.mf_cg_solve_host_workspace_bytes(d.op, 0), dtype=torch.uint8, device="cuda")
    sth = mf.mf_cg_solve_host(d.op, bh.data_ptr(), xh.data_ptr(), 1e-9, 2000, 0, ws.data_ptr(), ws.numel())
    assert sth["iterations"] == st["iterations"] and sth["rel_residual"] == st["rel_residual"]
    assert np.array_equal(xh.double().numpy(), xc)
    d.close()


@pytest.mark.parametrize("dims,k,geom,kind,prec,bc,ratio", [
    ((7, 6, 5), 3, "curved", mf.MF_LAPLACE, mf.MF_FP64, 1, 0.0),
    ((9, 5, 3), 2, "cart", mf.MF_HELMHOLTZ, mf.MF_FP64, 0, 10.0),
    ((6, 5, 4), 4, "shear", mf.MF_LAPLACE, mf.MF_FP64, 1, 100.0),
    ((7, 6, 5), 3, "curved", mf.MF_LAPLACE, mf.MF_FP32, 1, 0.0),
])
def test_chebyshev_jacobi_pcg_solves_oracle_equations(oracle, dims, k, geom, kind, prec, bc, ratio):
    """CG preconditioned by the degree-3 Chebyshev-accelerated Jacobi method (Sec. 5.2,
    Eqs. (chebyshev_weights), (chebyshev_richardson)): the solution satisfies the oracle's
    equations, and it takes fewer CG iterations than the unpreconditioned solver."""
    d = DevOp(*dims, k, geom, kind, 1.0, prec, bc)
    bu = inputs.random_unique(*dims, k, 19)
    b = d.native_from_unique(bu)
    rtol = 1e-5 if prec == mf.MF_FP32 else 1e-11
    x = torch.zeros(d.n_native, dtype=d.dtype, device="cuda")
    ws = torch.empty(mf.mf_cg_workspace_bytes_ex(d.op, 0, mf.MF_PRECOND_CHEBYSHEV), dtype=torch.uint8, device="cuda")
    st = mf.mf_cg_solve(d.op, b.data_ptr(), x.data_ptr(), rtol, 5000, 0, ws.data_ptr(), ws.numel(),
                        precond=mf.MF_PRECOND_CHEBYSHEV, cheb_ratio=ratio)
    assert st["code"] == mf.MF_OK and st["rel_residual"] <= rtol
    o = oracle_op(oracle, *dims, k, geom, 1.0 if kind == mf.MF_HELMHOLTZ else 0.0, bc)
    bm = np.where(o.boundary_mask(), 0.0, bu) if bc else bu
    if prec == mf.MF_FP32:
        bm = np.where(o.boundary_mask(), 0.0, bu.astype(np.float32).astype(np.float64)) if bc else bu
    res = np.linalg.norm(bm - o.apply(d.unique_from_native(x))) / np.linalg.norm(bm)
    assert res <= (1e-4 if prec == mf.MF_FP32 else 2e-11), res
    _, st0, _ = solve(d, b, rtol, 5000, 0)
    assert st["iterations"] < st0["iterations"], (st["iterations"], st0["iterations"])
    d.close()
