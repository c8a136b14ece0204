"""The 1D tables of the CUDA path, computed on the host by mf_tables.cpp, against textbook
routines: GLL nodes as the roots of (1 - x^2) P_k'(x), the Gauss rule of numpy's leggauss,
Lagrange values and derivatives from numpy polynomials through the nodes, the 1D mass and
stiffness matrices integrated exactly with a higher-order rule, and the fast diagonalisation
of (K, M) against scipy's generalised symmetric eigensolver (W W^T = M, W diag(lam) W^T = K,
the eigenvalues, every mode symmetric or antisymmetric, symmetric modes first).  Degrees
1..8; tests/tables_check.cpp prints the tables (a host program, no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_04534_gb300", "csrc")


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = tmp_path_factory.mktemp("tables") / "tables_check"
    src = [os.path.join(ROOT, "tests", "tables_check.cpp"), os.path.join(CSRC, "mf_tables.cpp")]
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                        *src], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0
    t = {}
    for line in out.stdout.splitlines():
        f = line.split()
        t[(f[0], int(f[1]))] = np.array([float(v) for v in f[2:]])
    return t


def lagrange(nodes):
    """numpy polynomials of the Lagrange basis through the nodes, and their derivatives."""
    n = len(nodes)
    P = []
    for i in range(n):
        others = np.delete(nodes, i)
        p = np.polynomial.Polynomial.fromroots(others)
        P.append(p / p(nodes[i]))
    return P, [p.deriv() for p in P]


@pytest.mark.parametrize("k", range(1, 9))
def test_nodes_rule_and_basis(tables, k):
    n = k + 1
    leg = np.polynomial.legendre.Legendre.basis(k)
    inner = np.sort(leg.deriv().roots().real) if k > 1 else np.array([])
    gll = 0.5 * (np.concatenate([[-1.0], inner, [1.0]]) + 1.0)
    np.testing.assert_allclose(tables[("nodes", k)], gll, atol=1e-14)
    xg, wg = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(tables[("qx", k)], 0.5 * (xg + 1.0), atol=1e-14)
    np.testing.assert_allclose(tables[("qw", k)], 0.5 * wg, atol=1e-14)
    P, dP = lagrange(gll)
    q = 0.5 * (xg + 1.0)
    S = np.array([[P[i](x) for i in range(n)] for x in q])
    D = np.array([[dP[i](x) for i in range(n)] for x in q])
    np.testing.assert_allclose(tables[("S", k)].reshape(n, n), S, atol=1e-12)
    np.testing.assert_allclose(tables[("D", k)].reshape(n, n), D, atol=1e-10 * np.abs(D).max())
    Pq, dPq = lagrange(q)  # collocation derivative on the Gauss points
    Dc = np.array([[dPq[r](x) for r in range(n)] for x in q])
    np.testing.assert_allclose(tables[("Dc", k)].reshape(n, n), Dc, atol=1e-10 * np.abs(Dc).max())


@pytest.mark.parametrize("k", range(1, 9))
def test_mass_and_stiffness_exact(tables, k):
    n = k + 1
    gll = tables[("nodes", k)]
    P, dP = lagrange(gll)
    xe, we = np.polynomial.legendre.leggauss(n + 3)  # exact for degree 2k + 5
    x, w = 0.5 * (xe + 1.0), 0.5 * we
    M = np.array([[np.sum(w * P[i](x) * P[j](x)) for j in range(n)] for i in range(n)])
    K = np.array([[np.sum(w * dP[i](x) * dP[j](x)) for j in range(n)] for i in range(n)])
    np.testing.assert_allclose(tables[("M", k)].reshape(n, n), M, atol=1e-13)
    np.testing.assert_allclose(tables[("K", k)].reshape(n, n), K, atol=1e-11 * np.abs(K).max())


@pytest.mark.parametrize("k", range(1, 9))
def test_fast_diagonalisation(tables, k):
    import scipy.linalg

    n = k + 1
    M = tables[("M", k)].reshape(n, n)
    K = tables[("K", k)].reshape(n, n)
    W = tables[("W", k)].reshape(n, n)  # W[j, m]: node j of mode m
    lam = tables[("lam", k)]
    np.testing.assert_allclose(W @ W.T, M, atol=1e-14)
    np.testing.assert_allclose(W @ np.diag(lam) @ W.T, K, atol=2e-13 * np.abs(K).max())
    ref = scipy.linalg.eigh(K, M, eigvals_only=True)
    np.testing.assert_allclose(np.sort(lam), np.sort(ref), atol=1e-12 * max(1.0, ref.max()))
    assert abs(lam.min()) < 1e-12 * ref.max()  # the constants: K 1 = 0
    par = []
    for m in range(n):
        w = W[:, m]
        if np.allclose(w, w[::-1], atol=1e-14):
            par.append(0)
        else:
            np.testing.assert_allclose(w, -w[::-1], atol=1e-14)
            par.append(1)
    assert par == sorted(par), par  # symmetric modes first
    for p in (0, 1):
        lp = [lam[m] for m in range(n) if par[m] == p]
        assert lp == sorted(lp)
    assert par.count(0) == (n + 1) // 2
