"""Independent reference constructions used to pin the oracle (tests only).

- 1D mass / stiffness of the GLL Lagrange basis integrated exactly by numpy's own
  higher-order Legendre-Gauss rule (nodes from numpy's Legendre roots);
- brute-force sparse assembly sum_K P_K^T A_K P_K from the oracle's element matrices.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import legendre as npleg


def gll_nodes_numpy(k):
    r = np.sort(npleg.Legendre.basis(k).deriv().roots().real) if k > 1 else np.array([])
    return np.concatenate([[0.0], (r + 1) / 2, [1.0]])


def _lagrange_np(nodes, s):
    """Values and derivatives of the Lagrange basis on `nodes` at points s (numpy, product form)."""
    n = len(nodes)
    s = np.atleast_1d(s)
    V = np.ones((len(s), n))
    D = np.zeros((len(s), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            f = (s - nodes[m]) / (nodes[i] - nodes[m])
            D[:, i] = D[:, i] * f + V[:, i] / (nodes[i] - nodes[m])
            V[:, i] = V[:, i] * f
    return V, D


def exact_1d_mass_stiffness(k):
    """M_ij = int_0^1 phi_i phi_j, K_ij = int_0^1 phi_i' phi_j' (integrands of degree <= 2k)
    with numpy's own (k+6)-point Legendre-Gauss rule, which integrates them exactly; nodes
    from numpy's Legendre roots -- nothing shared with the oracle's tables."""
    nodes = gll_nodes_numpy(k)
    xr, wr = npleg.leggauss(k + 6)
    x, w = (xr + 1) / 2, wr / 2
    V, D = _lagrange_np(nodes, x)
    return V.T @ (w[:, None] * V), D.T @ (w[:, None] * D)


def assemble_csr(op, dirichlet=False):
    """sum_K P_K^T A_K P_K with the oracle's explicit element matrices, as scipy CSR."""
    dofs = op.cell_dofs()
    n3 = op.n ** 3
    rows, cols, vals = [], [], []
    c = 0
    for cz in range(op.nz):
        for cy in range(op.ny):
            for cx in range(op.nx):
                A = op.element_matrix(cx, cy, cz)
                d = dofs[c]
                rows.append(np.repeat(d, n3))
                cols.append(np.tile(d, n3))
                vals.append(A.ravel())
                c += 1
    N = op.n_unique
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
    if dirichlet:
        keep = sp.diags((~op.boundary_mask()).astype(float))
        M = (keep @ M @ keep).tocsr()
    return M


def probe_dense(op):
    """Dense matrix of the oracle's matrix-free apply by probing with unit vectors."""
    N = op.n_unique
    A = np.zeros((N, N))
    e = np.zeros(N)
    for g in range(N):
        e[:] = 0.0
        e[g] = 1.0
        A[:, g] = op.apply(e)
    return A


def solve_direct(op, b):
    """Dirichlet solve (P A P) u = P b with the brute-force assembled matrix (sparse LU)."""
    A = assemble_csr(op, dirichlet=True)
    free = ~op.boundary_mask()
    u = np.zeros(op.n_unique)
    u[free] = spla.spsolve(A[free][:, free].tocsc(), b[free])
    return u
