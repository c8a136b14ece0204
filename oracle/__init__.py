"""FP64 CPU oracle for the continuous Q_k operator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It wraps ``mf_oracle.c`` (plain C, compiled with gcc) through ctypes
and shares no code with the CUDA library.

Every function states the passage of the paper it follows in ``mf_oracle.c``.  The pins
that tie it to something other than itself live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

AFFINE, CURVED = 0, 1


def build(force: bool = False) -> str:
    """Compile mf_oracle.c into liboracle.so with gcc (OpenMP over cells only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("geom", C.c_int),
                ("A", C.c_double * 9), ("b", C.c_double * 3), ("amp", C.c_double)]


class _Op(C.Structure):
    _fields_ = [("mesh", _Mesh), ("k", C.c_int), ("cm", C.c_double), ("bc", C.c_int), ("nq", C.c_int)]


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, vp = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_void_p
        _lib.or_apply.argtypes = [C.POINTER(_Op), vp, vp, C.c_int]
        _lib.or_apply_cells.argtypes = [C.POINTER(_Op), vp, C.c_int64, vp, vp, C.c_int]
        _lib.or_element_matrix.argtypes = [C.POINTER(_Op), C.c_int, C.c_int, C.c_int, vp]
        _lib.or_cell_dofs.argtypes = [C.POINTER(_Op), vp]
        _lib.or_scatter.argtypes = [C.POINTER(_Op), vp, vp]
        _lib.or_assemble.argtypes = [C.POINTER(_Op), vp, vp]
        _lib.or_boundary_mask.argtypes = [C.POINTER(_Op), vp]
        _lib.or_n_unique.argtypes = [C.POINTER(_Op)]
        _lib.or_n_unique.restype = C.c_int64
        _lib.or_cg.argtypes = [C.POINTER(_Op), vp, vp, C.c_int, C.c_double, vp, C.c_int]
        _lib.or_rhs_manufactured.argtypes = [C.POINTER(_Op), C.c_double, C.c_int, vp]
        _lib.or_errors.argtypes = [C.POINTER(_Op), C.c_double, vp, C.c_int, d, d]
        _lib.or_interpolate_manufactured.argtypes = [C.POINTER(_Op), C.c_double, vp]
        _lib.or_node_positions.argtypes = [C.POINTER(_Op), vp]
        _lib.or_volume.argtypes = [C.POINTER(_Op), C.c_int]
        _lib.or_volume.restype = C.c_double
        _lib.or_cell_det.argtypes = [C.POINTER(_Mesh), C.c_int, C.c_int, C.c_int, vp]
        _lib.or_cell_det.restype = C.c_double
        _lib.or_gll_nodes.argtypes = [C.c_int, vp]
        _lib.or_gauss.argtypes = [C.c_int, vp, vp]
        _lib.or_lagrange.argtypes = [C.c_int, vp, C.c_double, vp, vp]
        _lib.or_max_threads.restype = C.c_int
        del d, i64
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def max_threads() -> int:
    return int(_L().or_max_threads())


# ------------------------------------------------------------------ 1D tables
def gll_nodes(k: int) -> np.ndarray:
    out = np.zeros(k + 1)
    if _L().or_gll_nodes(k, _p(out)):
        raise ValueError("degree out of range")
    return out


def gauss(n: int):
    x, w = np.zeros(n), np.zeros(n)
    if _L().or_gauss(n, _p(x), _p(w)):
        raise ValueError("bad n")
    return x, w


def lagrange(nodes: np.ndarray, s: float):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    phi, dphi = np.zeros(len(nodes)), np.zeros(len(nodes))
    _L().or_lagrange(len(nodes), _p(nodes), float(s), _p(phi), _p(dphi))
    return phi, dphi


# ------------------------------------------------------------------ operator
class Op:
    """Operator description: unit cube split into nx*ny*nz cells, mapped affinely
    (x = A xh + b) or by the curved map xh + amp*sin(pi xh1)sin(pi xh2)sin(pi xh3)."""

    def __init__(self, nx, ny, nz, k, geom=AFFINE, cm=0.0, bc=0, A=None, b=None, amp=0.1, nq=None):
        m = _Mesh()
        m.nx, m.ny, m.nz, m.geom = nx, ny, nz, geom
        A = np.eye(3) if A is None else np.asarray(A, dtype=np.float64)
        b = np.zeros(3) if b is None else np.asarray(b, dtype=np.float64)
        for i in range(9):
            m.A[i] = float(A.flat[i])
        for i in range(3):
            m.b[i] = float(b[i])
        m.amp = amp
        self._op = _Op()
        self._op.mesh = m
        self._op.k, self._op.cm, self._op.bc = k, cm, bc
        self._op.nq = (k + 1) if nq is None else nq
        self.nx, self.ny, self.nz, self.k = nx, ny, nz, k
        self.n = k + 1
        self.ncells = nx * ny * nz

    @property
    def ref(self):
        return C.byref(self._op)

    @property
    def n_unique(self) -> int:
        return int(_L().or_n_unique(self.ref))

    @property
    def n_cellwise(self) -> int:
        return self.ncells * self.n ** 3

    def apply(self, xu: np.ndarray, nthreads: int = 0) -> np.ndarray:
        xu = np.ascontiguousarray(xu, dtype=np.float64)
        assert xu.shape == (self.n_unique,)
        yu = np.zeros_like(xu)
        _L().or_apply(self.ref, _p(xu), _p(yu), nthreads)
        return yu

    def apply_cells(self, xcw: np.ndarray, cells, nthreads: int = 0) -> np.ndarray:
        """Local (split) results A_K x_K for the listed cells from a canonical cell-wise x."""
        xcw = np.ascontiguousarray(xcw, dtype=np.float64).reshape(-1)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((len(cells), self.n ** 3))
        _L().or_apply_cells(self.ref, _p(xcw), len(cells), _p(cells), _p(out), nthreads)
        return out

    def element_matrix(self, cx: int, cy: int, cz: int) -> np.ndarray:
        n3 = self.n ** 3
        A = np.zeros((n3, n3))
        _L().or_element_matrix(self.ref, cx, cy, cz, _p(A))
        return A

    def cell_dofs(self) -> np.ndarray:
        out = np.zeros((self.ncells, self.n ** 3), dtype=np.int64)
        _L().or_cell_dofs(self.ref, _p(out))
        return out

    def scatter(self, xu: np.ndarray) -> np.ndarray:
        xu = np.ascontiguousarray(xu, dtype=np.float64)
        out = np.zeros(self.n_cellwise)
        _L().or_scatter(self.ref, _p(xu), _p(out))
        return out

    def assemble(self, ycw: np.ndarray) -> np.ndarray:
        ycw = np.ascontiguousarray(ycw, dtype=np.float64).reshape(-1)
        out = np.zeros(self.n_unique)
        _L().or_assemble(self.ref, _p(ycw), _p(out))
        return out

    def boundary_mask(self) -> np.ndarray:
        out = np.zeros(self.n_unique, dtype=np.uint8)
        _L().or_boundary_mask(self.ref, _p(out))
        return out.astype(bool)

    def cg(self, b: np.ndarray, maxit: int, rtol: float = 0.0, nthreads: int = 0):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        hist = np.zeros(maxit + 1)
        it = _L().or_cg(self.ref, _p(b), _p(x), maxit, rtol, _p(hist), nthreads)
        if it < 0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        return x, hist[: it + 1]

    def rhs_manufactured(self, freq: float = 2.0, nqr: int | None = None) -> np.ndarray:
        out = np.zeros(self.n_unique)
        _L().or_rhs_manufactured(self.ref, freq, self.k + 3 if nqr is None else nqr, _p(out))
        return out

    def errors(self, uh: np.ndarray, freq: float = 2.0, nqr: int | None = None):
        uh = np.ascontiguousarray(uh, dtype=np.float64)
        l2, h1 = C.c_double(), C.c_double()
        _L().or_errors(self.ref, freq, _p(uh), self.k + 3 if nqr is None else nqr, C.byref(l2), C.byref(h1))
        return l2.value, h1.value

    def interpolate_manufactured(self, freq: float = 2.0) -> np.ndarray:
        out = np.zeros(self.n_unique)
        _L().or_interpolate_manufactured(self.ref, freq, _p(out))
        return out

    def node_positions(self) -> np.ndarray:
        out = np.zeros((self.n_unique, 3))
        _L().or_node_positions(self.ref, _p(out))
        return out

    def volume(self, nqr: int | None = None) -> float:
        return float(_L().or_volume(self.ref, self.k + 1 if nqr is None else nqr))

    def cell_det(self, cx, cy, cz, xi) -> float:
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        return float(_L().or_cell_det(C.byref(self._op.mesh), cx, cy, cz, _p(xi)))
