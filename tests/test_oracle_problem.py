"""Pins for oracle.problem: the tau pencil assembly in the T basis.

A tau solve whose exact solution is a polynomial of degree < N has a zero
tau term, so the discrete solution must equal the exact coefficients
(closed form, independent of the assembly).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla
import pytest

from oracle import bases
from oracle.problem import TauProblem


def _poisson(N, left_val, right_val):
    # u'' = f  ->  dz(u) - uz = 0,  dz(uz) = f,  u(0) = left, u(1) = right
    pr = TauProblem(["u", "uz"], N, 0.0, 1.0)
    pr.add_equation("u_def", L_terms=[("u", "dz", 1.0), ("uz", "I", -1.0)])
    pr.add_equation("poisson", L_terms=[("uz", "dz", 1.0)])
    pr.add_bc("u", "left", value=left_val)
    pr.add_bc("u", "right", value=right_val)
    return pr


@pytest.mark.parametrize("N", [8, 16, 33])
def test_poisson_polynomial_solution_is_exact(N):
    # u = z^4 - z + 2:  u(0) = 2, u(1) = 2,  u'' = 12 z^2
    pr = _poisson(N, 2.0, 2.0)
    z = bases.chebyshev_grid(N)
    f = bases.chebyshev_forward(12 * z ** 2, N)
    M, L = pr.pencil_matrices(0.0)
    rhs = pr.rhs_vector({"poisson": f}, 0.0)
    X = sla.solve(L.toarray(), rhs)
    u, uz = X[:N], X[N:]
    assert np.abs(u - bases.chebyshev_forward(z ** 4 - z + 2, N)).max() < 1e-12
    assert np.abs(uz - bases.chebyshev_forward(4 * z ** 3 - 1, N)).max() < 1e-12


def test_row_bookkeeping():
    N = 10
    pr = _poisson(N, 0.0, 0.0)
    M, L = pr.pencil_matrices(1.0)
    assert L.shape == (2 * N, 2 * N)
    assert M.nnz == 0
    # differential equations lose their last row: 2 (N - 1) + 2 boundary rows
    assert len(pr.rhs_vector({}, 1.0)) == 2 * N


def test_unbalanced_system_rejected():
    pr = _poisson(8, 0.0, 0.0)
    pr.add_bc("uz", "left", value=0.0)
    with pytest.raises(ValueError):
        pr.pencil_matrices(0.0)


def test_dense_and_sparse_lu_agree():
    # oracle-vs-oracle floor of the two LU paths on a Helmholtz pencil
    N = 48
    pr = TauProblem(["u", "uz"], N, 0.0, 1.0)
    pr.add_equation("u_def", L_terms=[("u", "dz", 1.0), ("uz", "I", -1.0)])
    pr.add_equation("h", M_terms=[("u", "I", 1.0)],
                    L_terms=[("u", "I", lambda k: 0.1 * k * k), ("uz", "dz", -0.1)])
    pr.add_bc("u", "left", value=1.0)
    pr.add_bc("u", "right", value=0.5)
    M, L = pr.pencil_matrices(3.0)
    A = M + 1e-2 * L
    rhs = np.random.default_rng(5).standard_normal(2 * N) * (1 + 0j)
    x1 = sla.lu_solve(sla.lu_factor(A.toarray()), rhs)
    x2 = spla.splu(A.tocsc()).solve(rhs)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-13
