"""Serving: continuous batching of CG solve requests on one GPU (mf_server / mf_batch_*).

Each request's result must be the same alone and in the mix (bitwise: its kernels, order of
operations and reductions do not depend on what else is running), reach the requested
residual, and match the oracle's solution of the same discrete problem."""
import time

import numpy as np
import pytest
import torch

import paper_2609_04534_gb300 as mf
from paper_2609_04534_gb300 import inputs
from tests._fem_ref import solve_direct
from tests._gpu import oracle_op

pytestmark = pytest.mark.gpu


def run(server, reqs, timeout=300.0):
    outs = [np.zeros(inputs.unique_count(r.nx, r.ny, r.nz, r.degree)) if r.x_out_host is None else None for r in reqs]
    for r, o in zip(reqs, outs):
        r.x_out_host = o.ctypes.data
    tickets = [mf.mf_batch_submit(server, r) for r in reqs]
    res = [None] * len(tickets)
    t0 = time.time()
    while any(x is None for x in res):
        for i, t in enumerate(tickets):
            if res[i] is None:
                res[i] = mf.mf_batch_poll(server, t)
        assert time.time() - t0 < timeout, "serving timed out"
        time.sleep(0.002)
    return res, outs


def make_server(arena_gb=2.0, slots=16, batching=0):
    arena = torch.empty(int(arena_gb * 2**30), dtype=torch.uint8, device="cuda")
    return mf.mf_server_create(arena.data_ptr(), arena.numel(), max_slots=slots, batching=batching), arena


MIX = [
    dict(nx=6, ny=6, nz=6, degree=3, geometry=mf.MF_CURVED_SIN, rhs=mf.MF_RHS_MANUFACTURED, mixed=1),
    dict(nx=4, ny=5, nz=3, degree=2, geometry=mf.MF_AFFINE, rhs=mf.MF_RHS_RANDOM, seed=5, mixed=1),
    dict(nx=8, ny=8, nz=8, degree=4, geometry=mf.MF_CURVED_SIN, rhs=mf.MF_RHS_MANUFACTURED, mixed=1),
    dict(nx=5, ny=5, nz=5, degree=6, geometry=mf.MF_AFFINE, rhs=mf.MF_RHS_MANUFACTURED, mixed=0),
    dict(nx=3, ny=7, nz=4, degree=5, geometry=mf.MF_CURVED_SIN, kind=mf.MF_HELMHOLTZ, rhs=mf.MF_RHS_RANDOM,
         seed=9, mixed=1),
    dict(nx=12, ny=12, nz=12, degree=2, geometry=mf.MF_AFFINE, rhs=mf.MF_RHS_MANUFACTURED, mixed=1),
]


def test_mix_results_equal_alone_and_converge(oracle):
    sv, arena = make_server()
    try:
        res_mix, x_mix = run(sv, [mf.make_request(**p) for p in MIX])
    finally:
        mf.mf_server_destroy(sv)
    for p, r, x in zip(MIX, res_mix, x_mix):
        assert r["status"] == mf.MF_OK, (p, r)
        assert r["rel_residual"] <= 1e-10
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        if p["rhs"] == mf.MF_RHS_MANUFACTURED:
            assert 0 < r["l2_error"] < 0.1
    # the same mix with every request on its own graph chunks (no batched launches): bitwise equal
    sv, arena = make_server(batching=-1)
    try:
        res_solo, x_solo = run(sv, [mf.make_request(**p) for p in MIX])
    finally:
        mf.mf_server_destroy(sv)
    for p, r, r1, x, x1 in zip(MIX, res_mix, res_solo, x_mix, x_solo):
        assert r1["status"] == mf.MF_OK
        assert r1["iterations"] == r["iterations"], p
        assert np.array_equal(x1, x), p
    # each request alone on a fresh server: bitwise the same solution
    for p, x in zip(MIX, x_mix):
        sv, arena = make_server(slots=1)
        try:
            (r1,), (x1,) = run(sv, [mf.make_request(**p)])
        finally:
            mf.mf_server_destroy(sv)
        assert r1["status"] == mf.MF_OK
        assert np.array_equal(x1, x), p
    # one request against the oracle (same discrete problem, direct sparse solve)
    p = MIX[1]
    o = oracle_op(oracle, p["nx"], p["ny"], p["nz"], p["degree"], "cart", 0.0, 1)
    b = inputs.random_unique(p["nx"], p["ny"], p["nz"], p["degree"], p["seed"])
    b[o.boundary_mask()] = 0.0
    xo = solve_direct(o, b)
    assert np.abs(x_mix[1] - xo).max() <= 1e-8 * np.abs(xo).max()


def test_batches_of_one_class_match_solo_solves():
    """Eight requests of one class (Q3 curved Laplace, mixed) of different sizes and seeds run in
    one continuous batch; each result equals the request solved alone, bitwise, and FP64 ones
    (double-float CG vectors) batch the same way."""
    reqs = [dict(nx=4 + i, ny=5, nz=3 + (i % 3), degree=3, geometry=mf.MF_CURVED_SIN, rhs=mf.MF_RHS_RANDOM,
                 seed=30 + i, mixed=i % 2) for i in range(8)]
    sv, arena = make_server(slots=16)
    try:
        res, xs = run(sv, [mf.make_request(**p) for p in reqs])
    finally:
        mf.mf_server_destroy(sv)
    for p, r, x in zip(reqs, res, xs):
        assert r["status"] == mf.MF_OK and r["rel_residual"] <= 1e-10
        sv1, arena1 = make_server(slots=1, batching=-1)
        try:
            (r1,), (x1,) = run(sv1, [mf.make_request(**p)])
        finally:
            mf.mf_server_destroy(sv1)
        assert r1["iterations"] == r["iterations"]
        assert np.array_equal(x1, x), p


def test_admission_by_memory_and_queueing():
    """An arena that holds only a few requests at a time: all still complete, the peak use
    never exceeds the arena, and requests are admitted as memory frees up."""
    arena = torch.empty(96 * 2**20, dtype=torch.uint8, device="cuda")
    sv = mf.mf_server_create(arena.data_ptr(), arena.numel(), max_slots=8)
    try:
        reqs = [mf.make_request(8, 8, 8, 3, geometry=mf.MF_CURVED_SIN, rhs=mf.MF_RHS_RANDOM, seed=i, mixed=1)
                for i in range(10)]
        res, _ = run(sv, reqs)
        st = mf.mf_server_stats(sv)
    finally:
        mf.mf_server_destroy(sv)
    assert all(r["status"] == mf.MF_OK for r in res)
    assert st["arena_peak"] <= st["arena_bytes"]
    assert st["completed"] == 10 and st["active"] == 0 and st["pending"] == 0
    per = res[0]["device_bytes"]
    assert st["arena_peak"] < 10 * per  # not all resident at once
    admits = sorted(r["t_admit"] for r in res)
    assert admits[-1] > min(r["t_done"] for r in res)  # someone waited for memory


def test_oversize_cancel_and_bounded_drain():
    """Host-side failure paths: a request that can never fit, an invalid request, a request
    cancelled in the queue, one cancelled while running, and a drain that gives up."""
    arena = torch.empty(2 * 2**30, dtype=torch.uint8, device="cuda")
    sv = mf.mf_server_create(arena.data_ptr(), arena.numel(), max_slots=1)
    try:
        with pytest.raises(mf.MfError) as e:
            mf.mf_batch_submit(sv, mf.make_request(96, 96, 96, 4, geometry=mf.MF_CURVED_SIN))
        assert e.value.code == mf.MF_ERR_OOM
        with pytest.raises(mf.MfError) as e:
            mf.mf_batch_submit(sv, mf.make_request(4, 4, 4, 12))
        assert e.value.code == mf.MF_ERR_ARG
        # ~14M DoFs at FP64, ~1 ms per iteration, a 1e-14 target it cannot reach soon
        long_req = mf.make_request(48, 48, 48, 4, geometry=mf.MF_CURVED_SIN, rtol=1e-14, maxit=10**6, mixed=0)
        t1 = mf.mf_batch_submit(sv, long_req)
        t2 = mf.mf_batch_submit(sv, mf.make_request(4, 4, 4, 2))
        mf.mf_batch_cancel(sv, t2)  # still queued behind t1 (one slot)
        with pytest.raises(mf.MfError) as e:
            mf.mf_server_drain(sv, 0.05)
        assert e.value.code == mf.MF_ERR_TIMEOUT
        mf.mf_batch_cancel(sv, t1)
        mf.mf_server_drain(sv, 60.0)
        r1, r2 = mf.mf_batch_poll(sv, t1), mf.mf_batch_poll(sv, t2)
        assert r1["status"] == mf.MF_ERR_CANCELLED and r2["status"] == mf.MF_ERR_CANCELLED
    finally:
        mf.mf_server_destroy(sv)


def test_large_curved_q6_request_reaches_1e_10():
    """The largest kind of request of the serving stream -- curved Q6 on 60^3 cells (74 M
    cell-wise DoFs), mixed precision -- reaches relative residual 1e-10 through the server
    (the FP64 outer residual keeps the defect correction's true residual below the target)."""
    sv, arena = make_server(arena_gb=40.0, slots=4)
    try:
        r = mf.make_request(60, 60, 60, 6, geometry=mf.MF_CURVED_SIN, rhs=mf.MF_RHS_MANUFACTURED, rtol=1e-10,
                            maxit=400000, mixed=1)
        t = mf.mf_batch_submit(sv, r)
        t0 = time.time()
        res = None
        while res is None:
            res = mf.mf_batch_poll(sv, t)
            assert time.time() - t0 < 240.0, "request timed out"
            time.sleep(0.01)
    finally:
        mf.mf_server_destroy(sv)
    assert res["status"] == mf.MF_OK, res
    assert res["rel_residual"] <= 1e-10, res
    assert res["n_cellwise"] == 60**3 * 7**3


def test_persistent_batch_loops_over_more_units_than_resident_ctas():
    """Twelve Q4 requests of 16 x 16 x 28..32 cells (240-256 tiles: at the batching cap), two
    CTA-sized units per tile in the FP32 inner solve, make batched applies of ~3000 units per
    class (affine, curved), more than the GPU holds at once: the persistent launch's CTAs
    each take several units of several requests.  Every result equals the request solved
    alone, bitwise."""
    reqs = [dict(nx=16, ny=16, nz=28 + 2 * (i % 3), degree=4, geometry=mf.MF_CURVED_SIN if i % 2 else mf.MF_AFFINE,
                 rhs=mf.MF_RHS_RANDOM, seed=60 + i, mixed=1) for i in range(12)]
    sv, arena = make_server(arena_gb=8.0, slots=16)
    try:
        res, xs = run(sv, [mf.make_request(**p) for p in reqs], timeout=600.0)
    finally:
        mf.mf_server_destroy(sv)
    for p, r in zip(reqs, res):
        assert r["status"] == mf.MF_OK and r["rel_residual"] <= 1e-10, (p, r)
    for i in (0, 1, 11):
        sv1, arena1 = make_server(arena_gb=2.0, slots=1, batching=-1)
        try:
            (r1,), (x1,) = run(sv1, [mf.make_request(**reqs[i])], timeout=600.0)
        finally:
            mf.mf_server_destroy(sv1)
        assert r1["iterations"] == res[i]["iterations"]
        assert np.array_equal(x1, xs[i]), reqs[i]
