"""GB300-native matrix-free Q_k operator: thin Python binding of the C ABI in include/mf.h.

Every function here only marshals arguments (ints for device pointers, ctypes structs) and
calls ``libmf.so``; every step of the apply, the duplicate summation and the solvers runs
in the library's CUDA kernels.  There is no CPU fallback: importing the binding without a
built library raises.  PyTorch, where used by callers, supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK, MF_ERR_ARG, MF_ERR_OOM, MF_ERR_CUDA = 0, -1, -2, -3
MF_ERR_NOT_CONVERGED, MF_ERR_BREAKDOWN, MF_ERR_TIMEOUT, MF_ERR_BUSY, MF_ERR_UNSUPPORTED = -4, -5, -6, -7, -8
MF_ERR_CANCELLED = -9
MF_RHS_MANUFACTURED, MF_RHS_RANDOM = 0, 1
MF_AFFINE, MF_CURVED_SIN = 0, 1
MF_LAPLACE, MF_HELMHOLTZ = 0, 1
MF_FP64, MF_FP32, MF_MIXED, MF_FP64_DFMA = 0, 1, 2, 3
MF_BC_NONE, MF_BC_DIRICHLET0 = 0, 1
MF_CG_DEFAULT, MF_CG_SPLIT_DUAL, MF_CG_ASSEMBLED, MF_CG_SPLIT_DUAL_FUSED = 0, 1, 2, 3
MF_PRECOND_NONE, MF_PRECOND_JACOBI, MF_PRECOND_CHEBYSHEV = 0, 1, 2
MF_VARIANT_TENSOR = 3
MF_VARIANT_SMALL_CTA = 4
MF_VARIANT_OCCUPANCY = 5

_STATUS = {0: "MF_OK", -1: "MF_ERR_ARG", -2: "MF_ERR_OOM", -3: "MF_ERR_CUDA", -4: "MF_ERR_NOT_CONVERGED",
           -5: "MF_ERR_BREAKDOWN", -6: "MF_ERR_TIMEOUT", -7: "MF_ERR_BUSY", -8: "MF_ERR_UNSUPPORTED",
           -9: "MF_ERR_CANCELLED"}


class MfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class mf_info(C.Structure):
    _fields_ = [("n_cellwise", C.c_int64), ("n_unique", C.c_int64), ("n_native", C.c_int64),
                ("n_cells", C.c_int64), ("degree", C.c_int32), ("n", C.c_int32), ("elem_bytes", C.c_int32),
                ("path", C.c_int32), ("geom_bytes", C.c_size_t), ("workspace_bytes", C.c_size_t),
                ("algorithmic_bytes_per_apply", C.c_double)]


class mf_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer_iterations", C.c_int32), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int32), ("check_every", C.c_int32)]


class mf_solve_options(C.Structure):
    _fields_ = [("inner_rtol", C.c_double), ("chunk_iterations", C.c_int32), ("max_outer", C.c_int32),
                ("cg_form", C.c_int32), ("precond", C.c_int32), ("cheb_ratio", C.c_double),
                ("mixed_restart", C.c_int32), ("reserved", C.c_int32)]


class mf_server_config(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("queue_capacity", C.c_int32), ("chunk_iterations", C.c_int32),
                ("autotune", C.c_int32), ("inner_rtol", C.c_double), ("batching", C.c_int32),
                ("mixed_restart", C.c_int32)]


class mf_request(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("degree", C.c_int32),
                ("kind", C.c_int32), ("geometry", C.c_int32), ("mass_coeff", C.c_double),
                ("curve_amp", C.c_double), ("rhs", C.c_int32), ("freq", C.c_double), ("seed", C.c_uint64),
                ("rtol", C.c_double), ("maxit", C.c_int32), ("mixed", C.c_int32),
                ("x_out_host", C.c_void_p)]


class mf_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("outer_iterations", C.c_int32),
                ("rel_residual", C.c_double), ("l2_error", C.c_double), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("latency", C.c_double),
                ("n_cellwise", C.c_int64), ("n_unique", C.c_int64), ("device_bytes", C.c_size_t)]


class mf_server_stats_t(C.Structure):
    _fields_ = [("pending", C.c_int64), ("active", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("arena_bytes", C.c_size_t), ("arena_used", C.c_size_t), ("arena_peak", C.c_size_t)]


_lib = None


def lib() -> C.CDLL:
    """Load libmf.so (built by ``paper_2609_04534_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmf.so not built at {LIB_PATH}: run `python -m paper_2609_04534_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, sz, i32, d = C.c_void_p, C.c_size_t, C.c_int, C.c_double
    L.mf_last_error.restype = C.c_char_p
    L.mf_mesh_create.argtypes = [i32, i32, i32, i32, C.POINTER(C.c_double), d, C.POINTER(vp)]
    L.mf_mesh_destroy.argtypes = [vp]
    L.mf_mesh_destroy.restype = None
    L.mf_operator_create.argtypes = [vp, i32, i32, d, i32, i32, C.POINTER(vp)]
    L.mf_operator_destroy.argtypes = [vp]
    L.mf_operator_destroy.restype = None
    L.mf_operator_info.argtypes = [vp, C.POINTER(mf_info)]
    L.mf_operator_setup.argtypes = [vp, vp, sz, vp]
    for nm in ("mf_to_native", "mf_from_native", "mf_scatter_unique", "mf_gather_unique", "mf_apply",
               "mf_apply_split", "mf_apply_stream_twin"):
        getattr(L, nm).argtypes = [vp, vp, vp, vp]
    L.mf_dss.argtypes = [vp, vp, vp]
    L.mf_apply_split_block.argtypes = [vp, i32, vp, vp, vp]
    L.mf_make_consistent.argtypes = [vp, vp, vp]
    L.mf_apply_host_workspace_bytes.argtypes = [vp]
    L.mf_apply_host_workspace_bytes.restype = sz
    L.mf_apply_host.argtypes = [vp, vp, vp, vp, sz, vp]
    L.mf_reduce_workspace_bytes.argtypes = [vp]
    L.mf_reduce_workspace_bytes.restype = sz
    L.mf_dot.argtypes = [vp, vp, vp, i32, vp, vp, sz, vp]
    L.mf_dot_noalloc.argtypes = [vp, vp, vp, i32, vp, vp]
    L.mf_operator_autotune.argtypes = [vp, vp, vp, i32, vp]
    L.mf_operator_set_variant.argtypes = [vp, i32]
    L.mf_operator_get_variant.argtypes = [vp]
    L.mf_operator_get_variant.restype = i32
    L.mf_device_error.argtypes = [i32]
    L.mf_device_error.restype = i32
    L.mf_manufactured_workspace_bytes.argtypes = [vp]
    L.mf_manufactured_workspace_bytes.restype = sz
    L.mf_rhs_manufactured.argtypes = [vp, d, vp, vp, sz, vp]
    L.mf_error_manufactured.argtypes = [vp, d, vp, vp, vp, sz, vp]
    L.mf_cg_workspace_bytes.argtypes = [vp, i32]
    L.mf_cg_workspace_bytes.restype = sz
    L.mf_cg_solve.argtypes = [vp, vp, vp, d, i32, i32, C.POINTER(mf_solve_stats), vp, sz, vp]
    L.mf_cg_record_history.argtypes = [vp, i32]
    L.mf_cg_solve_ex.argtypes = [vp, vp, vp, d, i32, i32, C.POINTER(mf_solve_options), C.POINTER(mf_solve_stats),
                                 vp, sz, vp]
    L.mf_cg_workspace_bytes_ex.argtypes = [vp, i32, C.POINTER(mf_solve_options)]
    L.mf_cg_workspace_bytes_ex.restype = sz
    L.mf_cg_solve_host_workspace_bytes.argtypes = [vp, i32]
    L.mf_cg_solve_host_workspace_bytes.restype = sz
    L.mf_cg_solve_host.argtypes = [vp, vp, vp, d, i32, i32, C.POINTER(mf_solve_stats), vp, sz, vp]
    L.mf_diagonal_workspace_bytes.argtypes = [vp]
    L.mf_diagonal_workspace_bytes.restype = sz
    L.mf_diagonal.argtypes = [vp, vp, vp, sz, vp]
    L.mf_dss_atomic_workspace_bytes.argtypes = [vp]
    L.mf_dss_atomic_workspace_bytes.restype = sz
    L.mf_dss_atomic.argtypes = [vp, vp, vp, sz, vp]
    L.mf_cg_profile.argtypes = [vp, vp, vp, i32, i32, vp, sz, vp, C.POINTER(C.c_double)]
    L.mf_server_create.argtypes = [C.POINTER(mf_server_config), vp, sz, C.POINTER(vp)]
    L.mf_batch_submit.argtypes = [vp, C.POINTER(mf_request), C.POINTER(C.c_uint64)]
    L.mf_batch_poll.argtypes = [vp, C.c_uint64, C.POINTER(mf_result)]
    L.mf_batch_cancel.argtypes = [vp, C.c_uint64]
    L.mf_server_drain.argtypes = [vp, d]
    L.mf_server_stats.argtypes = [vp, C.POINTER(mf_server_stats_t)]
    L.mf_server_destroy.argtypes = [vp]
    L.mf_server_destroy.restype = None
    _lib = L
    return L


def _check(code: int) -> int:
    if code != MF_OK:
        raise MfError(code, lib().mf_last_error().decode())
    return code


def last_error() -> str:
    return lib().mf_last_error().decode()


# ---------------------------------------------------------------- handles
def mf_mesh_create(nx: int, ny: int, nz: int, geometry: int = MF_AFFINE, affine_3x4=None, curve_amp: float = 0.1):
    h = C.c_void_p()
    arr = None
    if affine_3x4 is not None:
        vals = [float(v) for v in affine_3x4]
        assert len(vals) == 12
        arr = (C.c_double * 12)(*vals)
    _check(lib().mf_mesh_create(nx, ny, nz, geometry, arr, curve_amp, C.byref(h)))
    return h.value


def mf_mesh_destroy(mesh) -> None:
    lib().mf_mesh_destroy(mesh)


def mf_operator_create(mesh, degree: int, kind: int = MF_LAPLACE, mass_coeff: float = 1.0,
                       precision: int = MF_FP64, bc: int = MF_BC_NONE):
    h = C.c_void_p()
    _check(lib().mf_operator_create(mesh, degree, kind, mass_coeff, precision, bc, C.byref(h)))
    return h.value


def mf_operator_destroy(op) -> None:
    lib().mf_operator_destroy(op)


def mf_operator_info(op) -> dict:
    info = mf_info()
    _check(lib().mf_operator_info(op, C.byref(info)))
    return {f: getattr(info, f) for f, _ in mf_info._fields_}


def mf_operator_setup(op, workspace_ptr: int, nbytes: int, stream: int = 0) -> None:
    _check(lib().mf_operator_setup(op, workspace_ptr or None, nbytes, stream or None))


def mf_operator_autotune(op, x_ptr: int, y_ptr: int, reps: int = 3, stream: int = 0) -> int:
    _check(lib().mf_operator_autotune(op, x_ptr, y_ptr, reps, stream or None))
    return int(lib().mf_operator_get_variant(op))


def mf_operator_set_variant(op, variant: int) -> None:
    _check(lib().mf_operator_set_variant(op, variant))


def mf_device_error(reset: bool = True) -> int:
    """The library's device error word (nonzero: a bounded wait in a kernel gave up)."""
    return int(lib().mf_device_error(1 if reset else 0))


def mf_operator_get_variant(op) -> int:
    return int(lib().mf_operator_get_variant(op))


# ---------------------------------------------------------------- vectors
def mf_to_native(op, canonical_ptr: int, native_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_to_native(op, canonical_ptr, native_ptr, stream or None))


def mf_from_native(op, native_ptr: int, canonical_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_from_native(op, native_ptr, canonical_ptr, stream or None))


def mf_scatter_unique(op, unique_ptr: int, native_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_scatter_unique(op, unique_ptr, native_ptr, stream or None))


def mf_gather_unique(op, native_ptr: int, unique_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_gather_unique(op, native_ptr, unique_ptr, stream or None))


def mf_make_consistent(op, native_ptr: int, stream: int = 0) -> None:
    """In place: every copy of a shared node becomes the average of its copies."""
    _check(lib().mf_make_consistent(op, native_ptr, stream or None))


def mf_apply(op, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_apply(op, x_ptr, y_ptr, stream or None))


def mf_apply_split(op, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_apply_split(op, x_ptr, y_ptr, stream or None))


def mf_apply_stream_twin(op, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    """The apply kernel's memory accesses without its arithmetic; y receives a copy of x."""
    _check(lib().mf_apply_stream_twin(op, x_ptr, y_ptr, stream or None))


def mf_apply_split_block(op, cells_per_cta: int, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    """mf_apply_split of a degree-3 operator with B = cells_per_cta cells per CTA (4, 8, 16, 32)."""
    _check(lib().mf_apply_split_block(op, cells_per_cta, x_ptr, y_ptr, stream or None))


def mf_dss(op, y_ptr: int, stream: int = 0) -> None:
    _check(lib().mf_dss(op, y_ptr, stream or None))


def mf_apply_host_workspace_bytes(op) -> int:
    return int(lib().mf_apply_host_workspace_bytes(op))


def mf_apply_host(op, x_host_ptr: int, y_host_ptr: int, workspace_ptr: int, nbytes: int, stream: int = 0) -> None:
    _check(lib().mf_apply_host(op, x_host_ptr, y_host_ptr, workspace_ptr, nbytes, stream or None))


def mf_reduce_workspace_bytes(op) -> int:
    return int(lib().mf_reduce_workspace_bytes(op))


def mf_dot(op, a_ptr: int, b_ptr: int, result_ptr: int, scratch_ptr: int, scratch_bytes: int, split: int = 0,
           stream: int = 0) -> None:
    _check(lib().mf_dot(op, a_ptr, b_ptr, split, result_ptr, scratch_ptr, scratch_bytes, stream or None))


def mf_dot_noalloc(op, a_ptr: int, b_ptr: int, result_ptr: int, split: int = 0, stream: int = 0) -> None:
    """mf_dot without caller scratch (static device scratch inside libmf; see include/mf.h)."""
    _check(lib().mf_dot_noalloc(op, a_ptr, b_ptr, split, result_ptr, stream or None))


def mf_manufactured_workspace_bytes(op) -> int:
    return int(lib().mf_manufactured_workspace_bytes(op))


def mf_rhs_manufactured(op, freq: float, b_ptr: int, scratch_ptr: int, scratch_bytes: int, stream: int = 0) -> None:
    _check(lib().mf_rhs_manufactured(op, freq, b_ptr, scratch_ptr, scratch_bytes, stream or None))


def mf_error_manufactured(op, freq: float, u_ptr: int, l2sq_ptr: int, scratch_ptr: int, scratch_bytes: int,
                          stream: int = 0) -> None:
    _check(lib().mf_error_manufactured(op, freq, u_ptr, l2sq_ptr, scratch_ptr, scratch_bytes, stream or None))


def mf_cg_workspace_bytes(op, mixed: int = 0) -> int:
    return int(lib().mf_cg_workspace_bytes(op, mixed))


def mf_cg_workspace_bytes_ex(op, mixed: int = 0, precond: int = 0) -> int:
    opts = mf_solve_options(0.0, 0, 0, 0, precond, 0.0, 0, 0)
    return int(lib().mf_cg_workspace_bytes_ex(op, mixed, C.byref(opts)))


def mf_cg_solve(op, b_ptr: int, x_ptr: int, rtol: float, maxit: int, mixed: int, workspace_ptr: int,
                nbytes: int, stream: int = 0, allow_not_converged: bool = False, inner_rtol: float = 0.0,
                chunk_iterations: int = 0, max_outer: int = 0, cg_form: int = 0, precond: int = 0,
                cheb_ratio: float = 0.0, mixed_restart: int = 0) -> dict:
    st = mf_solve_stats()
    opts = mf_solve_options(inner_rtol, chunk_iterations, max_outer, cg_form, precond, cheb_ratio, mixed_restart, 0)
    code = lib().mf_cg_solve_ex(op, b_ptr, x_ptr, rtol, maxit, mixed, C.byref(opts), C.byref(st), workspace_ptr,
                                nbytes, stream or None)
    if not (code == MF_OK or (allow_not_converged and code == MF_ERR_NOT_CONVERGED)):
        _check(code)
    out = {f: getattr(st, f) for f, _ in mf_solve_stats._fields_}
    out["code"] = code
    return out


def mf_cg_solve_host_workspace_bytes(op, mixed: int = 0) -> int:
    return int(lib().mf_cg_solve_host_workspace_bytes(op, mixed))


def mf_cg_solve_host(op, b_host_ptr: int, x_host_ptr: int, rtol: float, maxit: int, mixed: int, workspace_ptr: int,
                     nbytes: int, stream: int = 0, allow_not_converged: bool = False) -> dict:
    """CG from host memory: canonical b in, canonical x out (see include/mf.h)."""
    st = mf_solve_stats()
    code = lib().mf_cg_solve_host(op, b_host_ptr, x_host_ptr, rtol, maxit, mixed, C.byref(st), workspace_ptr, nbytes,
                                  stream or None)
    if not (code == MF_OK or (allow_not_converged and code == MF_ERR_NOT_CONVERGED)):
        _check(code)
    out = {f: getattr(st, f) for f, _ in mf_solve_stats._fields_}
    out["code"] = code
    return out


def mf_diagonal_workspace_bytes(op) -> int:
    return int(lib().mf_diagonal_workspace_bytes(op))


def mf_diagonal(op, diag_ptr: int, scratch_ptr: int, nbytes: int, stream: int = 0) -> None:
    _check(lib().mf_diagonal(op, diag_ptr, scratch_ptr, nbytes, stream or None))


def mf_dss_atomic_workspace_bytes(op) -> int:
    return int(lib().mf_dss_atomic_workspace_bytes(op))


def mf_dss_atomic(op, y_ptr: int, scratch_ptr: int, nbytes: int, stream: int = 0) -> None:
    _check(lib().mf_dss_atomic(op, y_ptr, scratch_ptr, nbytes, stream or None))


def mf_cg_profile(op, b_ptr: int, x_ptr: int, iterations: int, cg_form: int, workspace_ptr: int, nbytes: int,
                  stream: int = 0) -> dict:
    """Mean kernel durations (ms) of `iterations` directly launched CG iterations."""
    ms = (C.c_double * 4)()
    _check(lib().mf_cg_profile(op, b_ptr, x_ptr, iterations, cg_form, workspace_ptr, nbytes, stream or None, ms))
    return {"apply_ms": ms[0], "dss_ms": ms[1], "vector_ms": ms[2], "iteration_ms": ms[3]}


def mf_cg_record_history(hist_ptr: int | None, cap: int) -> None:
    _check(lib().mf_cg_record_history(hist_ptr, cap))


# ---------------------------------------------------------------- serving
def mf_server_create(arena_ptr: int, arena_bytes: int, max_slots: int = 32, queue_capacity: int = 0,
                     chunk_iterations: int = 0, autotune: int = 0, inner_rtol: float = 0.0, batching: int = 0,
                     mixed_restart: int = 0):
    cfg = mf_server_config(max_slots, queue_capacity, chunk_iterations, autotune, inner_rtol, batching, mixed_restart)
    h = C.c_void_p()
    _check(lib().mf_server_create(C.byref(cfg), arena_ptr, arena_bytes, C.byref(h)))
    return h.value


def make_request(nx, ny, nz, degree, kind=MF_LAPLACE, geometry=MF_AFFINE, mass_coeff=1.0, curve_amp=0.1,
                 rhs=MF_RHS_MANUFACTURED, freq=2.0, seed=0, rtol=1e-10, maxit=200000, mixed=1, x_out_ptr=None):
    return mf_request(nx, ny, nz, degree, kind, geometry, mass_coeff, curve_amp, rhs, freq, seed, rtol, maxit, mixed,
                      x_out_ptr)


def mf_batch_submit(server, req: mf_request) -> int:
    t = C.c_uint64()
    _check(lib().mf_batch_submit(server, C.byref(req), C.byref(t)))
    return int(t.value)


def mf_batch_poll(server, ticket: int):
    """Returns None while the request is pending, else a dict of its mf_result."""
    r = mf_result()
    code = lib().mf_batch_poll(server, ticket, C.byref(r))
    if code == MF_ERR_BUSY:
        return None
    _check(code)
    return {f: getattr(r, f) for f, _ in mf_result._fields_}


def mf_batch_cancel(server, ticket: int) -> None:
    _check(lib().mf_batch_cancel(server, ticket))


def mf_server_drain(server, timeout_s: float) -> None:
    _check(lib().mf_server_drain(server, timeout_s))


def mf_server_stats(server) -> dict:
    st = mf_server_stats_t()
    _check(lib().mf_server_stats(server, C.byref(st)))
    return {f: getattr(st, f) for f, _ in mf_server_stats_t._fields_}


def mf_server_destroy(server) -> None:
    lib().mf_server_destroy(server)
