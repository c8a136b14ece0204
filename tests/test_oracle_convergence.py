"""Manufactured-solution convergence of the oracle discretisation (pins the whole pipeline:
basis, quadrature, Jacobians of the affine and curved maps, assembly, Dirichlet, RHS and
error integrals).  Model problem of Sec. 2 / Sec. 6.1: -Lap u + c_m u = f on the unit cube
with homogeneous Dirichlet data; u = sin(2 pi x) sin(2 pi y) sin(2 pi z), so that
f = (12 pi^2 + c_m) u.  c_m = 0 is the Laplace problem; c_m = 1 the Helmholtz operator
(mass + Laplace, coefficient 1.0) of the degree sweep."""
import math

import numpy as np
import pytest

from tests._fem_ref import solve_direct

# (degree, map, meshes): the observed rate on the last two refinements must be within 0.2
# of k+1 (L2) and k (H1).
CASES = [
    (1, "cart", (4, 8, 16)),
    (2, "cart", (2, 4, 8)),
    (3, "cart", (2, 4, 8)),
    (1, "curved", (4, 8, 16)),
    (2, "curved", (2, 4, 8)),
    (3, "curved", (4, 6, 8)),
]


@pytest.mark.parametrize("cm", [0.0, 1.0], ids=["laplace", "helmholtz"])
@pytest.mark.parametrize("k,geom,Ns", CASES)
def test_manufactured_convergence_rates(oracle, k, geom, Ns, cm):
    l2s, h1s = [], []
    for N in Ns:
        op = oracle.Op(N, N, N, k, oracle.CURVED if geom == "curved" else oracle.AFFINE, cm=cm, bc=1)
        b = op.rhs_manufactured(2.0)
        u = solve_direct(op, b)
        l2, h1 = op.errors(u, 2.0)
        l2s.append(l2)
        h1s.append(h1)
    r_l2 = math.log(l2s[-2] / l2s[-1]) / math.log(Ns[-1] / Ns[-2])
    r_h1 = math.log(h1s[-2] / h1s[-1]) / math.log(Ns[-1] / Ns[-2])
    assert abs(r_l2 - (k + 1)) < 0.2, (l2s, r_l2)
    assert abs(r_h1 - k) < 0.2, (h1s, r_h1)


@pytest.mark.parametrize("geom", ["cart", "curved"])
@pytest.mark.parametrize("cm", [0.0, 1.0, 2.5])
def test_load_vector_sums_to_integral_of_f(oracle, geom, cm):
    """The basis is a partition of unity, so without Dirichlet masking the entries of the
    load vector b_i = int f phi_i sum to int_Omega f.  With u = sin(pi x) sin(pi y) sin(pi z)
    (frequency 1) and f = (3 pi^2 + c_m) u, int_Omega f = (3 pi^2 + c_m) (2/pi)^3 in closed
    form; the curved map sends the unit cube onto itself, so the value is the same there.  A
    dropped, mis-signed or mis-scaled mass term c_m shifts the sum by c_m (2/pi)^3, about
    3% of it per unit of c_m."""
    op = oracle.Op(4, 4, 4, 3, oracle.CURVED if geom == "curved" else oracle.AFFINE, cm=cm, bc=0)
    b = op.rhs_manufactured(1.0)
    exact = (3.0 * math.pi**2 + cm) * (2.0 / math.pi) ** 3
    assert abs(b.sum() / exact - 1.0) < 1e-10, (b.sum(), exact)


def test_oracle_cg_matches_direct_solve(oracle):
    op = oracle.Op(3, 3, 3, 2, oracle.CURVED, bc=1)
    b = op.rhs_manufactured(1.0)
    ud = solve_direct(op, b)
    uc, hist = op.cg(b, maxit=500, rtol=1e-13)
    assert hist[-1] <= 1e-13
    assert np.abs(uc - ud).max() < 1e-11 * np.abs(ud).max()
    # residual history is monotone in the A-norm sense only; the Euclidean one need not be,
    # but it must start at 1 and end below the tolerance
    assert hist[0] == 1.0


def test_interpolant_error_rate(oracle):
    """Nodal interpolation of the smooth u converges at k+1 in L2 on the curved mesh."""
    errs = []
    for N in (4, 8):
        op = oracle.Op(N, N, N, 2, oracle.CURVED)
        errs.append(op.errors(op.interpolate_manufactured(1.0), 1.0)[0])
    assert abs(math.log2(errs[0] / errs[1]) - 3.0) < 0.3
