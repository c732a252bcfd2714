"""Pins for oracle.bases: transforms and operator matrices.

Each check compares against something other than the oracle's own formula:
brute-force sums, numpy.polynomial.chebyshev (Clenshaw evaluation and
recurrences written independently of cos(n arccos x)), closed-form
expansions, and trigonometric definitions of U_n.
"""
import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

from oracle import bases

RNG = np.random.default_rng(1234)


# --- Fourier (Sec. "Fourier basis") -----------------------------------------

def test_fourier_forward_single_modes_closed_form():
    L, Ng, Nc = 4.0, 24, 16
    x = bases.fourier_grid(Ng, L)
    k = 2 * np.pi / L
    g = 0.7 + 3.0 * np.cos(2 * k * x) - 5.0 * np.sin(5 * k * x)
    f = bases.fourier_forward(g, Nc)
    expect = np.zeros(Nc // 2, complex)
    expect[0] = 0.7
    expect[2] = 1.5            # 3 cos -> 3/2 e^{ikx} + c.c.
    expect[5] = 2.5j           # -5 sin = -5 (e^{ikx} - e^{-ikx})/(2i) -> +2.5 i
    assert np.allclose(f, expect, atol=1e-14)


def test_fourier_forward_matches_brute_force_dft():
    L, Ng, Nc = 2 * np.pi, 12, 8
    g = RNG.standard_normal(Ng)
    f = bases.fourier_forward(g, Nc)
    x = bases.fourier_grid(Ng, L)
    for n in range(Nc // 2):
        s = sum(g[i] * np.exp(-1j * n * x[i]) for i in range(Ng)) / Ng
        assert abs(f[n] - s) < 1e-14


def test_fourier_backward_matches_brute_force_sum():
    L, Ng, Nc = 3.0, 18, 12
    f = RNG.standard_normal(Nc // 2) + 1j * RNG.standard_normal(Nc // 2)
    f[0] = f[0].real
    g = bases.fourier_backward(f, Ng)
    x = bases.fourier_grid(Ng, L)
    ks = bases.fourier_wavenumbers(Nc, L)
    for i in range(Ng):
        s = f[0].real + sum(2 * (f[n] * np.exp(1j * ks[n] * x[i])).real for n in range(1, Nc // 2))
        assert abs(g[i] - s) < 1e-13


def test_fourier_round_trip_dealiased():
    Nc, Ng = 32, 48
    f = RNG.standard_normal(Nc // 2) + 1j * RNG.standard_normal(Nc // 2)
    f[0] = f[0].real
    f2 = bases.fourier_forward(bases.fourier_backward(f, Ng), Nc)
    assert np.abs(f2 - f).max() < 1e-14


def test_fourier_product_equals_truncated_convolution():
    # quadratic product on the 3/2 grid = exact truncated convolution
    Nc, Ng = 16, 24
    K = Nc // 2
    a = RNG.standard_normal(K) + 1j * RNG.standard_normal(K); a[0] = a[0].real
    b = RNG.standard_normal(K) + 1j * RNG.standard_normal(K); b[0] = b[0].real
    prod = bases.fourier_forward(bases.fourier_backward(a, Ng) * bases.fourier_backward(b, Ng), Nc)
    full = lambda c: {**{n: c[n] for n in range(K)}, **{-n: np.conj(c[n]) for n in range(1, K)}}
    A, B = full(a), full(b)
    for n in range(K):
        s = sum(A[m] * B[n - m] for m in A if (n - m) in B)
        assert abs(prod[n] - s) < 1e-13


# --- Chebyshev (Sec. "Chebyshev basis") --------------------------------------

def test_chebyshev_grid_is_gauss_nodes():
    # roots of T_N, ascending: compare with numpy's chebpts1 (also the roots)
    for N in (8, 24, 48):
        assert np.allclose(bases.chebyshev_native_grid(N), np.sort(C.chebpts1(N)), atol=1e-15)


def test_chebyshev_backward_matches_clenshaw():
    Nc, Ng = 20, 30
    c = RNG.standard_normal(Nc)
    g = bases.chebyshev_backward(c, Ng)
    assert np.abs(g - C.chebval(bases.chebyshev_native_grid(Ng), c)).max() < 1e-13


def test_chebyshev_forward_closed_form_x_cubed():
    # x^3 = (3 T_1 + T_3) / 4
    Ng = 12
    x = bases.chebyshev_native_grid(Ng)
    c = bases.chebyshev_forward(x ** 3, 8)
    assert np.allclose(c, [0, 0.75, 0, 0.25, 0, 0, 0, 0], atol=1e-15)


@pytest.mark.parametrize("Nc,Ng", [(16, 16), (16, 24), (32, 48), (7, 11)])
def test_chebyshev_forward_recovers_polynomials(Nc, Ng):
    c = RNG.standard_normal(Nc)
    g = C.chebval(bases.chebyshev_native_grid(Ng), c)
    assert np.abs(bases.chebyshev_forward(g, Nc) - c).max() < 1e-13


def test_chebyshev_complex_data():
    Nc, Ng = 10, 15
    c = RNG.standard_normal(Nc) + 1j * RNG.standard_normal(Nc)
    g = bases.chebyshev_backward(c, Ng)
    assert np.abs(g.real - C.chebval(bases.chebyshev_native_grid(Ng), c.real)).max() < 1e-13
    assert np.abs(bases.chebyshev_forward(g, Nc) - c).max() < 1e-13


def test_chebyshev_dealiased_product_identity():
    # T_n T_j = (T_{n+j} + T_{|n-j|}) / 2 is exact in the first N_c coefficients
    # when 2 N_g > 3 (N_c - 1) (Appendix "Non-constant coefficients", dealiasing rule)
    Nc = 16
    Ng = 24
    assert 2 * Ng > 3 * (Nc - 1)
    for (n, j) in [(3, 5), (9, 12), (15, 15), (0, 7), (10, 14)]:
        en = np.eye(Nc)[n]; ej = np.eye(Nc)[j]
        prod = bases.chebyshev_forward(bases.chebyshev_backward(en, Ng) * bases.chebyshev_backward(ej, Ng), Nc)
        expect = np.zeros(2 * Nc)
        expect[n + j] += 0.5
        expect[abs(n - j)] += 0.5
        assert np.abs(prod - expect[:Nc]).max() < 1e-14


def test_chebyshev_product_aliases_without_padding():
    # at scale 1 the same product aliases into the kept coefficients
    Nc = 16
    en = np.eye(Nc)[9]; ej = np.eye(Nc)[12]
    prod = bases.chebyshev_forward(bases.chebyshev_backward(en, Nc) * bases.chebyshev_backward(ej, Nc), Nc)
    expect = np.zeros(Nc); expect[3] = 0.5
    assert np.abs(prod - expect).max() > 0.1


# --- operator matrices (Appendix) ---------------------------------------------

def _U(n, x):
    th = np.arccos(x)
    return np.sin((n + 1) * th) / np.sin(th)


def test_D_TT_matches_chebder():
    N = 14
    c = RNG.standard_normal(N)
    d = bases.cheb_D_TT(N) @ c
    ref = np.zeros(N); ref[: N - 1] = C.chebder(c)
    assert np.abs(d - ref).max() < 1e-12


def test_D_TU_derivative_in_U_basis():
    N = 12
    c = RNG.standard_normal(N)
    du = bases.cheb_D_TU(N) @ c
    x = np.linspace(-0.95, 0.95, 17)
    lhs = sum(du[i] * _U(i, x) for i in range(N))
    rhs = C.chebval(x, C.chebder(c))
    assert np.abs(lhs - rhs).max() < 1e-11


def test_P_L_conversion_to_U_basis():
    N = 12
    c = RNG.standard_normal(N)
    cu = bases.cheb_P_L(N) @ c
    x = np.linspace(-0.95, 0.95, 17)
    lhs = sum(cu[i] * _U(i, x) for i in range(N))
    assert np.abs(lhs - C.chebval(x, c)).max() < 1e-12


def test_P_R_dirichlet_basis():
    N = 10
    ct = RNG.standard_normal(N)
    c = bases.cheb_P_R(N) @ ct
    x = np.linspace(-1, 1, 13)
    D = lambda n: C.chebval(x, np.eye(N)[n]) - (C.chebval(x, np.eye(N)[n - 2]) if n >= 2 else 0)
    lhs = sum(ct[n] * D(n) for n in range(N))
    assert np.abs(C.chebval(x, c) - lhs).max() < 1e-12
    for n in range(2, N):
        assert abs(D(n)[0]) < 1e-14 and abs(D(n)[-1]) < 1e-14


def test_endpoint_and_integral_vectors():
    N = 9
    c = RNG.standard_normal(N)
    assert abs(bases.cheb_left_vector(N) @ c - C.chebval(-1.0, c)) < 1e-13
    assert abs(bases.cheb_right_vector(N) @ c - C.chebval(1.0, c)) < 1e-13
    ci = C.chebint(c, lbnd=-1)
    assert abs(bases.cheb_integrate_vector(N) @ c - C.chebval(1.0, ci)) < 1e-13


def test_derivative_on_problem_interval():
    # d/dz on [0, 1]: z = (x + 1)/2 -> factor 2
    N = 10
    z = bases.chebyshev_grid(N, 0.0, 1.0)
    c = bases.chebyshev_forward(z ** 4 - 2 * z, N)
    d = bases.chebyshev_derivative(c, 0.0, 1.0)
    assert np.abs(bases.chebyshev_backward(d, N) - (4 * z ** 3 - 2)).max() < 1e-12


@pytest.mark.parametrize("Nc,Ng", [(16, 24), (32, 48), (12, 12)])
def test_dct_variant_equals_quadrature(Nc, Ng):
    # the floor-estimate variant computes the same definition (scipy DCT)
    c = RNG.standard_normal((3, Nc)) + 1j * RNG.standard_normal((3, Nc))
    g = bases.chebyshev_backward(c, Ng)
    assert np.abs(bases.chebyshev_backward_dct(c, Ng) - g).max() < 1e-12   # O(N eps) sums
    assert np.abs(bases.chebyshev_forward_dct(g, Nc) - bases.chebyshev_forward(g, Nc)).max() < 1e-12
