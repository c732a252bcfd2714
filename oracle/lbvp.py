"""Linear boundary value solve and a potential-vorticity inversion with a
non-constant coefficient (oracle; test infrastructure).

Sec. "Linear boundary value solver": for every pencil, L_p X_p = F_p with
F_p the left-preconditioned right-hand side and the boundary values; here
each pencil is solved densely (the plain T-basis system of oracle.problem).

The workload (a reading: the paper solves a quasi-geostrophic inversion with
a stratification profile but prints no equations for it): on Fourier(x) x
Chebyshev(z in [0, 1]), given the potential vorticity q, find the stream
function psi with

    psiz_def:  dz(psi) - psiz = 0
    pv:        dx dx psi + dz(S(z) psiz) = q

S(z) = 1/N^2(z) a smooth stratification given by its Chebyshev coefficients
(a non-constant coefficient: Sec. "Non-constant coefficients"), rigid walls
psiz(0) = psiz(1) = 0, and in the k_x = 0 pencil (where the Neumann problem
fixes psi only up to a constant) psi(1) = 0 in place of psiz(1) = 0.

Pins: ``tests/test_oracle_lbvp.py`` (the NCC matrix against numpy's
Chebyshev series product, and a polynomial stream function recovered
exactly from its closed-form potential vorticity).
"""
import numpy as np
import scipy.linalg as sla

from .problem import NCC, TauProblem

QG_VARIABLES = ("psi", "psiz")


def qg_problem(n_z, strat):
    """The PV-inversion pencil problem; ``strat`` = Chebyshev coefficients of
    S(z) on [0, 1] (in T_n(2z - 1))."""
    pr = TauProblem(QG_VARIABLES, n_z, 0.0, 1.0)
    pr.add_equation("psiz_def", L_terms=[("psi", "dz", 1.0), ("psiz", "I", -1.0)])
    pr.add_equation("pv", L_terms=[("psi", "I", lambda k: -k * k), ("psiz", NCC(strat, "dz"), 1.0)])
    pr.add_bc("psiz", "left", value=0.0)
    pr.add_bc("psiz", "right", value=0.0, condition=lambda k: k != 0)
    pr.add_bc("psi", "right", value=0.0, condition=lambda k: k == 0)
    return pr


def solve_lbvp(problem, kx, F):
    """X[var, p, n] solving L_p X_p = F~_p for every pencil (dense LU);
    F maps equation name -> [p, n] T coefficients."""
    kx = np.asarray(kx, dtype=np.float64)
    S, N = problem.S, problem.N
    X = np.zeros((S, len(kx), N), dtype=np.complex128)
    for p, k in enumerate(kx):
        _, L = problem.pencil_matrices(k)
        rhs = problem.rhs_vector({e: F[e][p] for e in F}, k)
        X[:, p, :] = sla.solve(L.toarray(), rhs).reshape(S, N)
    return X
