"""Pins for the non-constant-coefficient operators and the linear boundary
value solve of the oracle (oracle.problem.ncc_matrix, oracle.lbvp).

* the NCC multiplication matrix applied to the Chebyshev coefficients of u
  equals numpy's Chebyshev series product g u truncated to N modes (an
  independent implementation of the same identity);
* a polynomial stream function psi = cos(k x) phi(z) with phi'(0) = phi'(1)
  = 0 and phi(1) = 0, and its potential vorticity q = -k^2 psi + dz(S dz psi)
  computed with numpy's polynomial algebra: the LBVP returns psi and
  psiz = dz psi exactly (to rounding) for every wavenumber, k_x = 0 included;
* dropping the NCC term's derivative or using S = 1 in place of S(z) is
  detected (the pin separates the operators).
"""
import numpy as np
import numpy.polynomial.chebyshev as C
from numpy.polynomial import Chebyshev, Polynomial
import pytest

from oracle import lbvp
from oracle.problem import ncc_matrix

L_X = 2 * np.pi


def test_ncc_matrix_is_the_truncated_series_product():
    rng = np.random.default_rng(0)
    N = 24
    for deg in (0, 1, 3, 6):
        g = rng.standard_normal(deg + 1)
        u = rng.standard_normal(N)
        full = C.chebmul(g, u)
        want = np.zeros(N)
        want[: min(N, len(full))] = full[:N]
        assert np.abs(ncc_matrix(g, N) @ u - want).max() < 1e-13


def _cheb01(poly_z, N):
    c = Polynomial(poly_z).convert(kind=Chebyshev, domain=[0.0, 1.0]).coef
    out = np.zeros(N)
    out[: len(c)] = c
    return out


# S(z) = 1 + z + z^2 / 2 ; phi(z) = 2 z^3 - 3 z^2 + 1 (phi'(0) = phi'(1) = 0, phi(1) = 0)
S_Z = [1.0, 1.0, 0.5]
PHI = [1.0, 0.0, -3.0, 2.0]


def _closed_form(N, kx, strat_z=S_Z):
    phi = Polynomial(PHI)
    dphi = phi.deriv()
    S = Polynomial(strat_z)
    P = len(kx)
    psi = np.zeros((P, N), complex)
    psiz = np.zeros((P, N), complex)
    q = np.zeros((P, N), complex)
    for p, k in enumerate(kx):
        amp = 1.0 if p == 0 else 0.5            # cos(k x) -> 1/2 e^{ikx} for k > 0
        qz = -k * k * phi + (S * dphi).deriv()
        psi[p] = amp * _cheb01(phi.coef, N)
        psiz[p] = amp * _cheb01(dphi.coef, N)
        q[p] = amp * _cheb01(qz.coef, N)
    return psi, psiz, q


@pytest.mark.parametrize("N", [8, 16, 32])
def test_lbvp_recovers_polynomial_stream_function(N):
    kx = 2 * np.pi * np.arange(5) / L_X
    strat = _cheb01(S_Z, 3)
    pr = lbvp.qg_problem(N, strat)
    psi, psiz, q = _closed_form(N, kx)
    X = lbvp.solve_lbvp(pr, kx, {"pv": q})
    assert np.abs(X[0] - psi).max() < 1e-12
    assert np.abs(X[1] - psiz).max() < 1e-12


def test_lbvp_pin_separates_the_ncc():
    N = 16
    kx = 2 * np.pi * np.arange(3) / L_X
    psi, psiz, q = _closed_form(N, kx)
    X = lbvp.solve_lbvp(lbvp.qg_problem(N, _cheb01([1.0], 3)), kx, {"pv": q})   # S = 1 instead of S(z)
    assert np.abs(X[0] - psi).max() > 1e-3
