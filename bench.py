"""Benchmark of the matrix-free Q_k hot path on GB300 (prints ONE JSON line on rank 0).

Workload (N=1): Q4 Laplace on the curved 64^3 mesh of the unit cube (x + 0.1 sin(pi x)
sin(pi y) sin(pi z) on every coordinate, per-Gauss-point Jacobians), FP64, homogeneous
Dirichlet.  A step is one CG iteration: q = P A P p (sum-factorised apply + deterministic
duplicate summation + mask) and the fused CG vector updates with their dot products.
value = cell-wise DoFs per step / step time; roofline = the CG apply's algorithmic bytes over
its time against the measured HBM bandwidth; e2e = the same K iterations through the C-ABI
host-buffer solve.  Extra fields: the applies of the curved 64^3 config (Q3/Q4, FP64 / FP64
on the native FP64 pipe / FP32), the Helmholtz degree sweep at ~50M cell-wise DoFs with the
per-degree HBM fractions, the 96^3 mixed-precision solve against plain FP64 CG, a burst of the
serving stream, and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-sweep]
                  [--no-solve] [--serve-burst NREQ] [--solve] [--serve NREQ --rate R]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "operator-apply GDoF/s and % HBM roofline per degree; solved DoF/s + p99 latency at 1e-10"
SWEEP_N = {1: 184, 2: 123, 3: 92, 4: 74, 5: 61, 6: 53, 7: 46, 8: 41}


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        p = {"hbm_gbs": float(j["hbm_gbs"]), "source": "measured"}
    except Exception:
        pass
    return p


class Clocks:
    """nvidia-smi sampling (every 100 ms) around the timed region; samples are timestamped and
    only those inside [mark_start, mark_end] are summarised (all of them if none fall inside)."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.t0 = self.t1 = None
        self.lines = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        time.sleep(1.0)  # nvidia-smi takes a moment before its first sample
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        import datetime

        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t1 is not None and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        for r in use:
            for nm, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": use[-1][2], "reasons": sorted(reasons),
                "samples": len(use), "window": "timed region" if inside else "whole run (none inside the timed region)"}


def aggregate_ranks(dist, device, t_local: float, units_local: float):
    """Replicas: every rank runs the same workload on its own GPU.  The job time is the max
    over ranks (after a barrier); the job throughput is the units all ranks processed / that
    time.  Works with any process group (NCCL on GPUs, gloo on CPU)."""
    import torch

    if dist is None:
        return t_local, units_local / t_local
    world = dist.get_world_size()
    tt = torch.tensor([t_local, units_local], dtype=torch.float64, device=device)
    tmax = tt[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    units = tt[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    dist.barrier()
    del world
    return float(tmax.item()), float(units.item()) / float(tmax.item())


def make_op(mf, torch, N, k, geom, kind, prec, bc, stream, affine=None):
    mesh = mf.mf_mesh_create(N, N, N, geom, affine, 0.1)
    op = mf.mf_operator_create(mesh, k, kind, 1.0, prec, bc)
    info = mf.mf_operator_info(op)
    ws = torch.empty(max(info["workspace_bytes"], 256), dtype=torch.uint8, device="cuda")
    mf.mf_operator_setup(op, ws.data_ptr(), ws.numel(), stream)
    return mesh, op, info, ws


def autotune(mf, torch, op, x, stream):
    y = torch.empty_like(x)
    v = mf.mf_operator_autotune(op, x.data_ptr(), y.data_ptr(), 3, stream)
    del y
    return v


def random_native(mf, torch, op, info, N, k, seed, dtype, stream):
    from paper_2609_04534_gb300 import inputs

    u = torch.as_tensor(inputs.random_unique(N, N, N, k, seed), device="cuda").to(dtype)
    x = torch.empty(info["n_native"], dtype=dtype, device="cuda")
    mf.mf_scatter_unique(op, u.data_ptr(), x.data_ptr(), stream)
    return x


def time_apply(mf, torch, op, x, y, stream_obj, reps, warm):
    s = stream_obj.cuda_stream
    for _ in range(warm):
        mf.mf_apply(op, x.data_ptr(), y.data_ptr(), s)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream_obj.synchronize()
    ev[0].record(stream_obj)
    for _ in range(reps):
        mf.mf_apply(op, x.data_ptr(), y.data_ptr(), s)
    ev[1].record(stream_obj)
    ev[1].synchronize()
    return ev[0].elapsed_time(ev[1]) / 1e3 / reps


def time_kernels(mf, torch, op, x, y, stream_obj, reps):
    """Per-kernel device time of the apply's two kernels (split apply, duplicate summation)."""
    s = stream_obj.cuda_stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ta = td = 0.0
    for _ in range(reps):
        e[0].record(stream_obj)
        mf.mf_apply_split(op, x.data_ptr(), y.data_ptr(), s)
        e[1].record(stream_obj)
        mf.mf_dss(op, y.data_ptr(), s)
        e[2].record(stream_obj)
        e[2].synchronize()
        ta += e[0].elapsed_time(e[1]) / 1e3
        td += e[1].elapsed_time(e[2]) / 1e3
    return ta / reps, td / reps


def time_twin(mf, torch, op, x, y, stream_obj, reps):
    """Device time of the apply kernel's stream twin: its grid and global loads and stores,
    none of its arithmetic (the access pattern's ceiling)."""
    s = stream_obj.cuda_stream
    mf.mf_apply_stream_twin(op, x.data_ptr(), y.data_ptr(), s)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream_obj)
    for _ in range(reps):
        mf.mf_apply_stream_twin(op, x.data_ptr(), y.data_ptr(), s)
    e[1].record(stream_obj)
    e[1].synchronize()
    return e[0].elapsed_time(e[1]) / 1e3 / reps


def cpu_baseline(N, k, curved, kind_helm, target_s=12.0):
    """The FP64 oracle (as it stands) on a bounded sample of cells of the same mesh, all
    host threads; reports cell-wise DoF/s of its apply."""
    import oracle

    oracle.build()
    o = oracle.Op(N, N, N, k, oracle.CURVED if curved else oracle.AFFINE, cm=1.0 if kind_helm else 0.0, bc=1)
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(0)
    ncal = 256
    cells = np.sort(rng.choice(o.ncells, ncal, replace=False)).astype(np.int64)
    xcw = np.zeros(o.ncells * n3) if o.ncells * n3 < 6e7 else None
    if xcw is None:
        return None
    xcw[:] = rng.uniform(-1, 1, xcw.size)
    t0 = time.perf_counter()
    o.apply_cells(xcw, cells)
    dt = time.perf_counter() - t0
    m = int(min(o.ncells, max(ncal, ncal * target_s / max(dt, 1e-6))))
    cells = np.sort(rng.choice(o.ncells, m, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    o.apply_cells(xcw, cells)
    dt = time.perf_counter() - t0
    return {"value": m * n3 / dt / 1e9, "unit": "GDoF/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{m} of {o.ncells} cells of the same mesh (local quadrature-loop apply, FP64), {dt:.1f} s"}


def workload_config(ncw: int, world: int) -> dict:
    """The bench's workload, reported identically by both arms."""
    return {"workload": "Q4 Laplace curved 64^3 (x+0.1 sin(pi x)sin(pi y)sin(pi z)), per-Gauss-point "
                        "Jacobians, FP64, Dirichlet; step = one split-dual CG iteration (apply with <p,Ap> at "
                        "the quadrature points; DSS folded into the x/r update; p = r + beta p), "
                        "b uniform[-1,1] seed 1",
            "n_cellwise": ncw, "global_batch": 1, "seq_len": 0,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (vectors 262 MB + geometry 1.57 GB per apply)"}


def reference_arm(args):
    """CPU oracle arm: each step applies the oracle to a bounded sample of cells."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    N, k = 64, 4
    o = oracle.Op(N, N, N, k, oracle.CURVED, bc=1)
    n3 = (k + 1) ** 3
    rng = np.random.default_rng(0)
    xcw = rng.uniform(-1, 1, o.ncells * n3)
    m = 2048
    cells = np.sort(rng.choice(o.ncells, m, replace=False)).astype(np.int64)
    for _ in range(args.warmup):
        o.apply_cells(xcw, cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.apply_cells(xcw, cells)
    dt = (time.perf_counter() - t0) / args.steps
    v = m * n3 / dt / 1e9
    sample = f"{m} of {o.ncells} cells per step (local quadrature-loop apply, FP64)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(o.ncells * n3, 1),
            "cpu_baseline": {"value": v, "unit": "GDoF/s", "kind": "oracle", "cores": oracle.max_threads(),
                             "sample": sample + "; the oracle's apply stands for the CG step (the apply is its "
                                                "dominant part)"},
            "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_apply(args):
    """A few applies of one case, for ncu captures of the apply and DSS kernels."""
    import torch

    import paper_2609_04534_gb300 as mf

    N, k, geom, prec, kind = args.profile_apply.split(",")
    N, k = int(N), int(k)
    g = mf.MF_CURVED_SIN if geom == "curved" else mf.MF_AFFINE
    p = {"fp64": mf.MF_FP64, "fp32": mf.MF_FP32}[prec]
    kd = mf.MF_HELMHOLTZ if kind == "helmholtz" else mf.MF_LAPLACE
    dt = torch.float64 if p == mf.MF_FP64 else torch.float32
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    # geom "shear": a sheared affine map (the general path with one metric per mesh: the curved
    # kernel's arithmetic without its per-point metric stream)
    shear = [1.0, 0.3, 0.0, 0.1, 1.2, -0.2, 0.0, 0.25, 0.9, 0.0, 0.0, 0.0] if geom == "shear" else None
    mesh, op, info, ws = make_op(mf, torch, N, k, g, kd, p, 0, s, affine=shear)
    with torch.cuda.stream(stream):
        x = random_native(mf, torch, op, info, N, k, 1, dt, s)
        y = torch.empty_like(x)
    tensor = mf.mf_operator_get_variant(op) == mf.MF_VARIANT_TENSOR
    small = [mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY] if p == mf.MF_FP64 else []
    for v in ([args.variant] if args.variant >= 0 else [0, 1, 2] + small + ([mf.MF_VARIANT_TENSOR] if tensor else [])):
        mf.mf_operator_set_variant(op, v)
        t = time_apply(mf, torch, op, x, y, stream, args.reps, 1)
        ta, td = time_kernels(mf, torch, op, x, y, stream, args.reps)
        print(json.dumps({"case": args.profile_apply, "variant": v, "n_cellwise": info["n_cellwise"],
                          "ms": round(t * 1e3, 4), "gdofs": round(info["n_cellwise"] / t / 1e9, 3),
                          "apply_kernel_ms": round(ta * 1e3, 4), "dss_kernel_ms": round(td * 1e3, 4),
                          "apply_kernel_hbm_frac": round(info["algorithmic_bytes_per_apply"] / ta / 1e9 / peaks()["hbm_gbs"], 4)}),
              flush=True)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)


def profile_cg(args):
    """A few CG iterations of one case through mf_cg_profile (each kernel launched directly),
    for ncu captures of the CG kernels: the apply with <p, A p>, alpha, update, direction."""
    import torch

    import paper_2609_04534_gb300 as mf

    N, k, geom, prec = args.profile_cg.split(",")
    N, k = int(N), int(k)
    g = mf.MF_CURVED_SIN if geom == "curved" else mf.MF_AFFINE
    p = {"fp64": mf.MF_FP64, "fp32": mf.MF_FP32}[prec]
    dt = torch.float64 if p == mf.MF_FP64 else torch.float32
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    mesh, op, info, ws = make_op(mf, torch, N, k, g, mf.MF_LAPLACE, p, mf.MF_BC_DIRICHLET0, s)
    with torch.cuda.stream(stream):
        b = random_native(mf, torch, op, info, N, k, 1, dt, s)
        x = torch.zeros_like(b)
        cws = torch.empty(mf.mf_cg_workspace_bytes(op, 0), dtype=torch.uint8, device="cuda")
    stream.synchronize()
    r = mf.mf_cg_profile(op, b.data_ptr(), x.data_ptr(), args.reps, mf.MF_CG_SPLIT_DUAL, cws.data_ptr(),
                         cws.numel(), s)
    print(json.dumps({"case": args.profile_cg, "n_cellwise": info["n_cellwise"],
                      **{kk: round(v, 4) for kk, v in r.items()}}), flush=True)
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)


def dss_ablation(args):
    """Sec. 6 ablations: the deterministic layer-disjoint duplicate summation against an
    atomic one (one line per case), and the apply's launch variants (cells per CTA and
    resident CTAs per SM)."""
    import torch

    import paper_2609_04534_gb300 as mf

    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for N, k, geom, prec in ((64, 4, "curved", "fp64"), (64, 3, "curved", "fp64"), (64, 4, "curved", "fp32"),
                             (123, 2, "affine", "fp64")):
        g = mf.MF_CURVED_SIN if geom == "curved" else mf.MF_AFFINE
        p = {"fp64": mf.MF_FP64, "fp32": mf.MF_FP32}[prec]
        dt = torch.float64 if p == mf.MF_FP64 else torch.float32
        mesh, op, info, ws = make_op(mf, torch, N, k, g, mf.MF_LAPLACE, p, 0, s)
        with torch.cuda.stream(stream):
            x = random_native(mf, torch, op, info, N, k, 1, dt, s)
            y = torch.empty_like(x)
            sc = torch.empty(mf.mf_dss_atomic_workspace_bytes(op), dtype=torch.uint8, device="cuda")
        mf.mf_apply_split(op, x.data_ptr(), y.data_ptr(), s)
        out = {"case": f"Q{k} {geom} {N}^3 {prec}", "n_cellwise": info["n_cellwise"], "n_unique": info["n_unique"]}
        for name, fn in (("sweep_dss_ms", lambda: mf.mf_dss(op, y.data_ptr(), s)),
                         ("atomic_dss_ms", lambda: mf.mf_dss_atomic(op, y.data_ptr(), sc.data_ptr(), sc.numel(), s))):
            for _ in range(3):
                fn()
            stream.synchronize()
            ev[0].record(stream)
            for _ in range(args.reps):
                fn()
            ev[1].record(stream)
            ev[1].synchronize()
            out[name] = round(ev[0].elapsed_time(ev[1]) / args.reps, 4)
        out["atomic_over_sweep"] = round(out["atomic_dss_ms"] / out["sweep_dss_ms"], 3)
        variants = {}
        for v in (0, 1, 2):
            mf.mf_operator_set_variant(op, v)
            t = time_apply(mf, torch, op, x, y, stream, args.reps, 2)
            variants[f"variant{v}"] = {"apply_ms": round(t * 1e3, 4), "gdofs": round(info["n_cellwise"] / t / 1e9, 3)}
        out["apply_variants"] = variants
        print(json.dumps(out), flush=True)
        mf.mf_operator_destroy(op)
        mf.mf_mesh_destroy(mesh)
        del ws, x, y, sc
        torch.cuda.empty_cache()


def block_sweep(args):
    """Sec. 6 block-size sweep: the degree-3 split apply (no duplicate summation) with B = 4, 8,
    16, 32 cells per CTA, the resident threads per SM held at launch variant 0's, Laplace on
    N^3 cells (128^3: 134 M cell-wise DoFs, the paper's size), Cartesian and curved, FP64
    (double-float) and FP32; then the Cartesian Helmholtz FP64 apply of the ~50 M DoF degree
    sweep at k = 1..8.  Beside it: launch variants 0-2 and the operator's default (the
    tensor-core apply for Cartesian FP64 at k = 2, 3)."""
    import torch

    import paper_2609_04534_gb300 as mf

    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    N, k = args.block_n, 3
    pk = peaks()["hbm_gbs"]

    def timed(fn):
        for _ in range(3):
            fn()
        stream.synchronize()
        ev[0].record(stream)
        for _ in range(args.reps):
            fn()
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3 / args.reps

    # degree 3 on N^3 (every path and precision), then the Cartesian Helmholtz FP64 apply of
    # the ~50 M DoF degree sweep at every degree
    cases = [(N, 3, geom, prec, mf.MF_LAPLACE) for geom, prec in
             (("cart", "fp64"), ("curved", "fp64"), ("cart", "fp32"), ("curved", "fp32"))]
    if not args.no_sweep:
        cases += [(nn, kk, "cart", "fp64", mf.MF_HELMHOLTZ) for kk, nn in SWEEP_N.items()]
    for N, k, geom, prec, kind in cases:
        g = mf.MF_CURVED_SIN if geom == "curved" else mf.MF_AFFINE
        p = {"fp64": mf.MF_FP64, "fp32": mf.MF_FP32}[prec]
        dt = torch.float64 if p == mf.MF_FP64 else torch.float32
        mesh, op, info, ws = make_op(mf, torch, N, k, g, kind, p, 0, s)
        with torch.cuda.stream(stream):
            x = random_native(mf, torch, op, info, N, k, 1, dt, s)
            y = torch.empty_like(x)
        ab = info["algorithmic_bytes_per_apply"]
        out = {"case": f"Q{k} {'Helmholtz' if kind == mf.MF_HELMHOLTZ else 'Laplace'} {geom} {N}^3 {prec}",
               "n_cellwise": info["n_cellwise"], "algorithmic_bytes": ab}

        def rec(t):
            return {"ms": round(t * 1e3, 4), "gdofs": round(info["n_cellwise"] / t / 1e9, 3),
                    "hbm_frac": round(ab / t / 1e9 / pk, 4)}
        default = mf.mf_operator_get_variant(op)
        for b in (4, 8, 16, 32):
            if 32 <= (k + 1) ** 2 * b <= 1024:
                out[f"B{b}"] = rec(timed(lambda: mf.mf_apply_split_block(op, b, x.data_ptr(), y.data_ptr(), s)))
        dd_only = {mf.MF_VARIANT_SMALL_CTA, mf.MF_VARIANT_OCCUPANCY} if p == mf.MF_FP64 else set()
        for v in sorted({0, 1, 2, default} | dd_only):
            mf.mf_operator_set_variant(op, v)
            out[f"variant{v}"] = rec(timed(lambda: mf.mf_apply_split(op, x.data_ptr(), y.data_ptr(), s)))
        out["default_variant"] = default
        print(json.dumps(out), flush=True)
        mf.mf_operator_destroy(op)
        mf.mf_mesh_destroy(mesh)
        del ws, x, y
        torch.cuda.empty_cache()


def solve_compare(N=96, inner=(1e-3,), extra=True):
    """Mixed-precision Poisson solve: Q4 on the curved N^3 mesh (96^3 is the config), manufactured
    u = sin(2 pi x) sin(2 pi y) sin(2 pi z), FP32 apply inside FP64 defect correction to
    relative residual 1e-10, against plain FP64 CG (double-float apply) on the same problem.
    extra adds the Jacobi-preconditioned runs."""
    import torch

    import paper_2609_04534_gb300 as mf

    k = 4
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    out = {"metric": "solved DoF/s at relative residual 1e-10", "workload":
           f"Q4 Poisson curved {N}^3, manufactured sin(2 pi x)sin(2 pi y)sin(2 pi z), Dirichlet"}
    mesh, op, info, ws = make_op(mf, torch, N, k, mf.MF_CURVED_SIN, mf.MF_LAPLACE, mf.MF_MIXED, 1, s)
    # the plain FP64 solver runs on an MF_FP64 operator of the same mesh (double-float apply)
    mesh64, op64, _, ws64 = make_op(mf, torch, N, k, mf.MF_CURVED_SIN, mf.MF_LAPLACE, mf.MF_FP64, 1, s)
    b = torch.empty(info["n_native"], dtype=torch.float64, device="cuda")
    sc = torch.empty(mf.mf_manufactured_workspace_bytes(op), dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    mf.mf_rhs_manufactured(op, 2.0, b.data_ptr(), sc.data_ptr(), sc.numel(), s)
    stream.synchronize()
    out["rhs_setup_s"] = time.perf_counter() - t0
    x = torch.zeros_like(b)
    autotune(mf, torch, op, b, s)
    autotune(mf, torch, op64, b, s)
    l2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (mixed, inner tolerance, preconditioner, Chebyshev interval ratio b / a, restarted inner CG)
    runs = [(1, t, 0, 0.0, 0) for t in inner] + [(0, 0.0, 0, 0.0, 0)]
    if extra:
        runs += [(1, 0.0, 0, 0.0, 1)]
        runs += [(1, 0.0, mf.MF_PRECOND_JACOBI, 0.0, 0), (0, 0.0, mf.MF_PRECOND_JACOBI, 0.0, 0)]
        runs += [(0, 0.0, mf.MF_PRECOND_CHEBYSHEV, r, 0) for r in (10.0, 30.0, 100.0)]
    for mixed, itol, pre, ratio, restart in runs:
        sop = op if mixed else op64
        cws = torch.empty(mf.mf_cg_workspace_bytes_ex(sop, mixed, pre), dtype=torch.uint8, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        st = mf.mf_cg_solve(sop, b.data_ptr(), x.data_ptr(), 1e-10, 400000, mixed, cws.data_ptr(), cws.numel(), s,
                            allow_not_converged=True, inner_rtol=itol, precond=pre, cheb_ratio=ratio,
                            mixed_restart=restart)
        ev[1].record(stream)
        ev[1].synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        mf.mf_error_manufactured(op, 2.0, x.data_ptr(), l2.data_ptr(), sc.data_ptr(), sc.numel(), s)
        stream.synchronize()
        tag = {mf.MF_PRECOND_NONE: "", mf.MF_PRECOND_JACOBI: "_jacobi",
               mf.MF_PRECOND_CHEBYSHEV: f"_chebyshev{ratio:g}"}[pre]
        tag += "_restarted" if restart else ""
        out[((f"mixed_inner{itol:g}" if itol else "mixed") if mixed else "fp64") + tag] = {
            "status": st["code"], "iterations": st["iterations"], "outer": st["outer_iterations"],
            "rel_residual": st["rel_residual"], "seconds": t,
            "applies": st["iterations"] * (3 if pre == mf.MF_PRECOND_CHEBYSHEV else 1),
            "solved_gdofs_cellwise": info["n_cellwise"] / t / 1e9, "solved_gdofs_unique": info["n_unique"] / t / 1e9,
            "l2_error": float(l2.item()) ** 0.5}
        del cws
        torch.cuda.empty_cache()
    out["n_cellwise"], out["n_unique"] = info["n_cellwise"], info["n_unique"]
    best = min((v["seconds"], kk) for kk, v in out.items()
               if kk.startswith("mixed") and "jacobi" not in kk and "restarted" not in kk)
    out["best_mixed"] = best[1]
    out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / best[0]
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)
    mf.mf_operator_destroy(op64)
    mf.mf_mesh_destroy(mesh64)
    del ws, ws64, b, x, sc
    torch.cuda.empty_cache()
    return out


def solve_run(args):
    print(json.dumps(solve_compare(args.solve_n, tuple(args.inner_rtol), True)), flush=True)


def serve_stream(n, rate=0.0, single=False, no_batching=False, arena_gb=120, mixed_restart=0, nmax=64, chunk=0):
    """Serving stream: n Poisson CG solve requests, mesh N^3 with N log-uniform in [4, nmax],
    degree uniform in {2..6}, affine or curved 50/50, manufactured right-hand side, FP32 apply
    in FP64 refinement to 1e-10; seed 4.  Reports p50/p99 latency (submit -> result) and
    solved DoF/s over the makespan.  rate 0: all requests at t = 0 (a closed burst)."""
    import torch

    import paper_2609_04534_gb300 as mf

    rng = np.random.default_rng(4)
    Ns = np.rint(np.exp(rng.uniform(np.log(4), np.log(nmax), n))).astype(int)
    ks = rng.integers(2, 7, n)
    geo = rng.integers(0, 2, n)
    arena = torch.empty(int(arena_gb * 2**30), dtype=torch.uint8, device="cuda")
    # single: the baseline of the same stream, the plain FP64 solver one request at a time
    sv = mf.mf_server_create(arena.data_ptr(), arena.numel(), max_slots=1 if single else 64, autotune=1,
                             chunk_iterations=chunk,
                             batching=-1 if (no_batching or single) else 0, mixed_restart=mixed_restart)
    reqs = [mf.make_request(int(N), int(N), int(N), int(k), geometry=mf.MF_CURVED_SIN if g else mf.MF_AFFINE,
                            rhs=mf.MF_RHS_MANUFACTURED, rtol=1e-10, maxit=400000, mixed=0 if single else 1)
            for N, k, g in zip(Ns, ks, geo)]
    gaps = rng.exponential(1.0 / rate, n) if rate > 0 else np.zeros(n)
    t0 = time.perf_counter()
    tickets, results = [], {}
    nxt = 0.0
    for i, r in enumerate(reqs):
        nxt += gaps[i]
        while time.perf_counter() - t0 < nxt:
            time.sleep(0.0005)
        tickets.append(mf.mf_batch_submit(sv, r))
    while len(results) < n:
        for t in tickets:
            if t not in results:
                res = mf.mf_batch_poll(sv, t)
                if res is not None:
                    results[t] = res
        time.sleep(0.001)
    makespan = time.perf_counter() - t0
    st = mf.mf_server_stats(sv)
    mf.mf_server_destroy(sv)
    rs = [results[t] for t in tickets]
    lat = np.array([r["latency"] for r in rs])
    ok = [r for r in rs if r["status"] == 0]
    out = {"metric": "serving: solved DoF/s and p50/p99 latency at 1e-10", "requests": n,
           "arrival_rate_per_s": rate if rate > 0 else "all at t=0 (closed burst)", "ok": len(ok),
           "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
           "makespan_s": makespan,
           "solved_gdofs_cellwise": sum(r["n_cellwise"] for r in ok) / makespan / 1e9,
           "solved_gdofs_unique": sum(r["n_unique"] for r in ok) / makespan / 1e9,
           "max_rel_residual": max(r["rel_residual"] for r in ok) if ok else None,
           "status_counts": {str(k): int(v) for k, v in zip(*np.unique([r["status"] for r in rs], return_counts=True))},
           "failed": [dict(N=int(Ns[i]), k=int(ks[i]), curved=int(geo[i]), status=int(rs[i]["status"]),
                           iterations=int(rs[i]["iterations"]), outer=int(rs[i]["outer_iterations"]),
                           rel=float(rs[i]["rel_residual"])) for i in range(n) if rs[i]["status"] != 0][:10],
           "slowest": [dict(N=int(Ns[i]), k=int(ks[i]), curved=int(geo[i]), iterations=int(rs[i]["iterations"]),
                            outer=int(rs[i]["outer_iterations"]), latency_s=round(float(lat[i]), 3))
                       for i in np.argsort(-lat)[:5]],
           "inner_cg": "restarted" if mixed_restart else "reliable updates",
           "mesh_n_range": [4, nmax], "chunk_iterations": chunk or 10,
           "batching": not (no_batching or single),
           "solver": "plain FP64 CG, one request at a time" if single else "mixed precision, 64 slots",
           "arena_peak_gb": st["arena_peak"] / 2**30, "slots": 1 if single else 64}
    del arena
    torch.cuda.empty_cache()
    return out


def serve_run(args):
    print(json.dumps(serve_stream(args.serve, args.rate, args.fp64_single, args.no_batching,
                                  mixed_restart=int(args.mixed_restart), nmax=args.serve_nmax,
                                  chunk=args.serve_chunk)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the 96^3 mixed vs FP64 solve of the default line")
    ap.add_argument("--serve-burst", type=int, default=100,
                    help="requests of the serving burst in the default line (0: skip)")
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--profile-apply", default=None, metavar="N,k,geom,prec,kind",
                    help="only run a few applies of one case (for ncu), e.g. 32,4,curved,fp64,laplace")
    ap.add_argument("--profile-cg", default=None, metavar="N,k,geom,prec",
                    help="only run --reps CG iterations of one case (for ncu), e.g. 48,4,curved,fp64")
    ap.add_argument("--dss-ablation", action="store_true",
                    help="only time the sweep vs atomic duplicate summation and the apply's launch variants")
    ap.add_argument("--block-sweep", action="store_true",
                    help="Sec. 6 block-size sweep of the degree-3 apply (B = 4..32 cells per CTA)")
    ap.add_argument("--block-n", type=int, default=128, help="cells per axis of the --block-sweep mesh")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", type=int, default=-1, help="--profile-apply: launch variant (-1: all)")
    ap.add_argument("--serve", type=int, default=0, metavar="NREQ",
                    help="serving run: NREQ solve requests with Poisson arrivals (prints its own JSON line)")
    ap.add_argument("--rate", type=float, default=0.0, help="serving arrival rate (requests/s); 0 = measure capacity")
    ap.add_argument("--no-batching", action="store_true", help="serving: every request on its own graph chunks")
    ap.add_argument("--serve-nmax", type=int, default=64, help="serving: largest mesh N (N^3 cells)")
    ap.add_argument("--serve-chunk", type=int, default=0, help="serving: CG iterations per graph launch (0: 10)")
    ap.add_argument("--mixed-restart", action="store_true",
                    help="serving: restart the inner FP32 CG at every defect-correction step")
    ap.add_argument("--fp64-single", action="store_true",
                    help="serving baseline: the same stream through the plain FP64 solver, one request at a time")
    ap.add_argument("--solve-n", type=int, default=96, help="cells per axis of the --solve mesh")
    ap.add_argument("--inner-rtol", type=float, nargs="+", default=[0.0],
                    help="inner FP32 CG tolerances to run (0: the library default)")
    args = ap.parse_args()
    if args.profile_apply:
        profile_apply(args)
        return
    if args.profile_cg:
        profile_cg(args)
        return
    if args.dss_ablation:
        dss_ablation(args)
        return
    if args.block_sweep:
        block_sweep(args)
        return
    if args.solve:
        solve_run(args)
        return
    if args.serve:
        serve_run(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch

    import paper_2609_04534_gb300 as mf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pk = peaks()
    stream = torch.cuda.Stream()
    s = stream.cuda_stream

    # ------------------------------------------------------------ primary: CG iteration
    N, k = 64, 4
    mesh, op, info, ws = make_op(mf, torch, N, k, mf.MF_CURVED_SIN, mf.MF_LAPLACE, mf.MF_FP64, mf.MF_BC_DIRICHLET0, s)
    ncw = info["n_cellwise"]
    with torch.cuda.stream(stream):
        b = random_native(mf, torch, op, info, N, k, 1, torch.float64, s)
        x = torch.zeros_like(b)
        y = torch.empty_like(b)
        cws = torch.empty(mf.mf_cg_workspace_bytes(op, 0), dtype=torch.uint8, device="cuda")
    stream.synchronize()
    variant = autotune(mf, torch, op, b, s)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with Clocks(local) as clk:
        # warm-up (also builds and caches the solve's graph path once)
        mf.mf_cg_solve(op, b.data_ptr(), x.data_ptr(), 0.0, args.warmup, 0, cws.data_ptr(), cws.numel(), s,
                       allow_not_converged=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        ev[0].record(stream)
        st = mf.mf_cg_solve(op, b.data_ptr(), x.data_ptr(), 0.0, args.steps, 0, cws.data_ptr(), cws.numel(), s,
                            allow_not_converged=True)
        ev[1].record(stream)
        ev[1].synchronize()
        clk.mark_end()
    torch.cuda.synchronize()
    t_steps = ev[0].elapsed_time(ev[1]) / 1e3
    its = st["iterations"]
    t_steps, rate = aggregate_ranks(dist, "cuda", t_steps, float(ncw) * its)
    t_it = t_steps / max(its, 1)
    value = rate / 1e9

    # apply alone on the same operator, plus per-kernel times of the step's kernels: the CG
    # iteration launched kernel by kernel with CUDA events on the bench stream (both forms)
    t_apply = time_apply(mf, torch, op, b, y, stream, 20, 3)
    t_split, t_dss = time_kernels(mf, torch, op, b, y, stream, 10)
    t_twin = time_twin(mf, torch, op, b, y, stream, 20)
    prof = {}
    for form, nm in ((mf.MF_CG_SPLIT_DUAL, "split_dual"), (mf.MF_CG_SPLIT_DUAL_FUSED, "split_dual_fused_p"),
                     (mf.MF_CG_ASSEMBLED, "assembled")):
        prof[nm] = mf.mf_cg_profile(op, b.data_ptr(), x.data_ptr(), 20, form, cws.data_ptr(), cws.numel(), s)
    t_fused = prof["split_dual"]["apply_ms"] / 1e3
    alg_bytes = info["algorithmic_bytes_per_apply"]
    # Byte roofline of the step's dominant kernel, the CG apply (A_K p and <p, A_K p>): the
    # algorithmic bytes of one apply (x 8 + y 8 + 6 metric words x 8 = 64 B per cell-wise DoF
    # for the curved FP64 Laplace operator) over its CUDA-event time, against the measured HBM
    # copy bandwidth.  traffic: DRAM bytes of this kernel from one ncu capture of the same kernel
    # on the curved Q4 48^3 case, 78.4 B per cell-wise DoF (the 14.4 above 64: its next-wave
    # L2 prefetch), scaled to the bench's DoFs.
    traffic = 1084.3e6 / 13824000 * ncw
    roof = {"bound": "hbm", "achieved": alg_bytes / t_fused / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": alg_bytes / t_fused / 1e9 / pk["hbm_gbs"], "traffic": traffic,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy kernel), of measured" if pk["source"] == "measured"
            else "fallback 6800 GB/s",
            "algorithmic_bytes_per_dof": alg_bytes / ncw,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of apply_general<dd,dd,5,16,2,1,0> "
                              "on Q4 curved 48^3 (13.82 M DoFs): 1084.3 MB, scaled by DoFs; 874.6 MB with the "
                              "L2 prefetch off",
            "kernel": "apply_general<dd,dd,5,curved,laplace> as the split-dual CG apply "
                      "(A_K p and <p, A_K p> at the quadrature points)",
            "kernel_ms": round(t_fused * 1e3, 4),
            "dram_gbs_from_traffic": traffic / t_fused / 1e9,
            # the same accesses without the arithmetic (mf_apply_stream_twin): the layout's ceiling
            "twin_frac": alg_bytes / t_twin / 1e9 / pk["hbm_gbs"]}
    hbm_frac_apply = alg_bytes / t_apply / 1e9 / pk["hbm_gbs"]

    # e2e through the C ABI from host buffers: mf_cg_solve_host copies the canonical b from
    # pinned host memory, runs the same K iterations and copies the canonical x back, all
    # inside the timed call
    e2e = None
    try:
        ncan = info["n_cellwise"]
        can = torch.empty(ncan, dtype=torch.float64, device="cuda")
        mf.mf_from_native(op, b.data_ptr(), can.data_ptr(), s)
        hb = torch.empty(ncan, dtype=torch.float64, pin_memory=True)
        hb.copy_(can.cpu())
        hx = torch.empty(ncan, dtype=torch.float64, pin_memory=True)
        hws = torch.empty(mf.mf_cg_solve_host_workspace_bytes(op, 0), dtype=torch.uint8, device="cuda")
        del can
        mf.mf_cg_solve_host(op, hb.data_ptr(), hx.data_ptr(), 0.0, args.warmup, 0, hws.data_ptr(), hws.numel(), s,
                            allow_not_converged=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st2 = mf.mf_cg_solve_host(op, hb.data_ptr(), hx.data_ptr(), 0.0, args.steps, 0, hws.data_ptr(), hws.numel(),
                                  s, allow_not_converged=True)
        te = time.perf_counter() - t0
        its2 = max(st2["iterations"], 1)
        e2e = {"value": world * ncw * st2["iterations"] / te / 1e9, "unit": "GDoF/s",
               "h2d_bytes_per_step": ncan * 8 / its2, "d2h_bytes_per_step": ncan * 8 / its2,
               "note": "one mf_cg_solve_host call (C ABI, pinned host buffers in canonical layout): H2D of b, "
                       "layout conversion, K CG iterations, conversion back, D2H of x, synchronise; copies "
                       "amortised per step"}
        del hws, hb, hx
    except Exception as exc:  # keep the line even if pinned memory is unavailable
        e2e = {"value": None, "unit": "GDoF/s", "error": str(exc)[:200]}
    del cws
    mf.mf_operator_destroy(op)
    mf.mf_mesh_destroy(mesh)
    del ws, b, x, y
    torch.cuda.empty_cache()

    # ------------------------------------------------------------ applies of the same config
    applies = {}
    for kk in (3, 4):
        for prec, dt, nm in ((mf.MF_FP64, torch.float64, "fp64"), (mf.MF_FP64_DFMA, torch.float64, "fp64_dfma"),
                             (mf.MF_FP32, torch.float32, "fp32")):
            mesh, op, info, ws = make_op(mf, torch, 64, kk, mf.MF_CURVED_SIN, mf.MF_LAPLACE, prec, 0, s)
            with torch.cuda.stream(stream):
                xx = random_native(mf, torch, op, info, 64, kk, 1, dt, s)
                yy = torch.empty_like(xx)
            autotune(mf, torch, op, xx, s)
            t = time_apply(mf, torch, op, xx, yy, stream, 20, 3)
            ta, td = time_kernels(mf, torch, op, xx, yy, stream, 5)
            tt = time_twin(mf, torch, op, xx, yy, stream, 20)
            gd = info["n_cellwise"] / t / 1e9
            applies[f"Q{kk}_{nm}"] = {"gdofs": round(gd, 3),
                                      "hbm_frac": round(info["algorithmic_bytes_per_apply"] / t / 1e9 / pk["hbm_gbs"], 4),
                                      "apply_kernel_ms": round(ta * 1e3, 4), "dss_kernel_ms": round(td * 1e3, 4),
                                      "twin_kernel_ms": round(tt * 1e3, 4), "apply_over_twin": round(ta / tt, 3)}
            mf.mf_operator_destroy(op)
            mf.mf_mesh_destroy(mesh)
            del ws, xx, yy
            torch.cuda.empty_cache()

    # ------------------------------------------------------------ degree sweep (Helmholtz, ~50M)
    # mf_apply (local apply + duplicate summation) per degree with the autotuned launch variant
    # (variant 3: the tensor-core apply of degrees 1..3), against 16 B per cell-wise DoF
    sweep = {}
    frac_deg, kfrac_deg = {}, {}
    if not args.no_sweep:
        for kk, NN in SWEEP_N.items():
            ent = {"N": NN}
            for prec, nm in ((mf.MF_FP64, "fp64"), (mf.MF_FP64_DFMA, "fp64_dfma")):
                mesh, op, info, ws = make_op(mf, torch, NN, kk, mf.MF_AFFINE, mf.MF_HELMHOLTZ, prec, 0, s)
                with torch.cuda.stream(stream):
                    xx = random_native(mf, torch, op, info, NN, kk, 2, torch.float64, s)
                    yy = torch.empty_like(xx)
                v = autotune(mf, torch, op, xx, s)
                t = time_apply(mf, torch, op, xx, yy, stream, 10, 3)
                ta, td = time_kernels(mf, torch, op, xx, yy, stream, 5)
                gd = info["n_cellwise"] / t / 1e9
                ab = info["algorithmic_bytes_per_apply"]
                ent["n_cellwise"] = info["n_cellwise"]
                ent[nm] = {"gdofs": round(gd, 3), "hbm_frac": round(ab / t / 1e9 / pk["hbm_gbs"], 4),
                           "apply_kernel_ms": round(ta * 1e3, 4), "dss_kernel_ms": round(td * 1e3, 4),
                           "apply_kernel_hbm_frac": round(ab / ta / 1e9 / pk["hbm_gbs"], 4), "variant": v}
                if nm == "fp64":
                    frac_deg[f"k{kk}"] = ent[nm]["hbm_frac"]
                    kfrac_deg[f"k{kk}"] = ent[nm]["apply_kernel_hbm_frac"]
                mf.mf_operator_destroy(op)
                mf.mf_mesh_destroy(mesh)
                del ws, xx, yy
                torch.cuda.empty_cache()
            sweep[f"k{kk}"] = ent

    # ------------------------------------------------------------ the metric's second half
    # config 4: the mixed-precision solve against plain FP64 CG, to 1e-10 (each with its clocks)
    solve = None
    if rank == 0 and not args.no_solve:
        try:
            with Clocks(local) as sclk:
                sclk.mark_start()
                solve = solve_compare(args.solve_n, (0.0,), False)
                sclk.mark_end()
            solve["clocks"] = sclk.summary()
        except Exception as exc:
            solve = {"error": str(exc)[:200]}
    # config 5 (shortened): a burst of requests of the serving stream through the batched
    # mixed-precision server
    serve = serve_unbatched = None
    if rank == 0 and args.serve_burst > 0:
        try:
            with Clocks(local) as vclk:
                vclk.mark_start()
                serve = serve_stream(args.serve_burst, 0.0, False, False, arena_gb=60)
                vclk.mark_end()
            serve["clocks"] = vclk.summary()
        except Exception as exc:
            serve = {"error": str(exc)[:200]}
        # the same burst with every request on its own graph chunks (batching off)
        try:
            with Clocks(local) as uclk:
                uclk.mark_start()
                serve_unbatched = serve_stream(args.serve_burst, 0.0, False, True, arena_gb=60)
                uclk.mark_end()
            serve_unbatched["clocks"] = uclk.summary()
            serve_unbatched.pop("slowest", None)
        except Exception as exc:
            serve_unbatched = {"error": str(exc)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(64, 4, True, False)
        except Exception as exc:
            cpu = {"value": None, "error": str(exc)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "GDoF/s", "n_gpus": world, "steps": its,
            "warmup": args.warmup, "ms_per_step": round(t_it * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (double-float arithmetic on the FP32 pipe, ~2^-48; config-3 degrees 2-3: exact "
                     "integer digits on the FP16 tensor cores)",
            "data": "synthetic",
            "config": workload_config(ncw, world),
            "roofline": roof,
            "apply_hbm_frac_per_degree": frac_deg,
            "apply_kernel_hbm_frac_per_degree": kfrac_deg,
            "apply_only": {"gdofs": round(ncw / t_apply / 1e9, 4), "hbm_frac_of_measured": round(hbm_frac_apply, 4),
                           "apply_kernel_ms": round(t_split * 1e3, 4), "dss_kernel_ms": round(t_dss * 1e3, 4),
                           "twin_kernel_ms": round(t_twin * 1e3, 4),
                           "twin_hbm_frac_of_measured": round(alg_bytes / t_twin / 1e9 / pk["hbm_gbs"], 4)},
            "cg_iteration_kernels_ms": {k: {kk: round(vv, 4) for kk, vv in v.items()} for k, v in prof.items()},
            "apply_variant": variant,
            "applies_64cubed_curved": applies,
            "helmholtz_sweep_50M": sweep,
            "solve_96cubed": solve,
            "serve_burst": serve,
            "serve_burst_unbatched": serve_unbatched,
            "cpu_baseline": cpu,
            "e2e": e2e,
            # mask, max|b|, zero x, scale b, copy p, <r,r>, state; then 4 kernels per iteration
            # (apply, alpha, update, p) in graph chunks of 20 iterations (a partial last chunk
            # still launches its kernels); the final conversion of x
            "gpu_launches": 7 + 4 * 20 * ((its + 19) // 20) + 1,
            "clocks": clk.summary(),
            "peaks": pk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
