"""Pins for the advective terms of the Rayleigh-Benard oracles (2D and 3D).

The equations of the Rayleigh-Benard reading carry the right-hand sides
F_f = -(u dx f + v dy f + w fz) for f in (b, u, v, w) (v and dy in 3D only),
with the first-order fields fz entering directly.  A manufactured state made
of a few trigonometric-times-polynomial terms is band limited well inside the
dealiased grid (Sec. "Scaled transforms & dealiasing": products of modes below
N/2 are exact on the 3/2 grid), so the oracle's F must equal the closed form
pointwise to rounding.  The closed form is evaluated at random points; the
oracle's coefficients are summed there explicitly (Chebyshev series in
2z - 1 by numpy's chebval, Fourier sums written out), without the oracle's
transforms.  Every field of the state differs from every other, so a swapped
pairing (w uz in place of w wz), a dropped term or a flipped sign moves the
result by O(1).
"""
import numpy as np
from numpy.polynomial import Chebyshev, Polynomial
from numpy.polynomial import chebyshev as C

from oracle import rb, rb3d

TWO_PI = 2.0 * np.pi


def _cheb(poly_z, n_z):
    """Chebyshev coefficients in T_n(2z - 1) of a polynomial in z (ascending powers)."""
    c = Polynomial(poly_z).convert(kind=Chebyshev, domain=[0.0, 1.0]).coef
    out = np.zeros(n_z)
    out[: len(c)] = c
    return out


def _poly(poly_z, z):
    return Polynomial(poly_z)(z)


# A field is a list of terms (amplitude, 'cos'|'sin', m_x, m_y, z polynomial):
# amplitude * trig(m_x x + m_y y) * q(z) on the 2 pi periodic box.
def _eval(terms, x, y, z):
    out = np.zeros_like(x)
    for a, kind, mx, my, q in terms:
        th = mx * x + my * y
        out += a * (np.cos(th) if kind == "cos" else np.sin(th)) * _poly(q, z)
    return out


def _dx(terms):
    out = []
    for a, kind, mx, my, q in terms:
        if mx:
            out.append((-a * mx, "sin", mx, my, q) if kind == "cos" else (a * mx, "cos", mx, my, q))
    return out


def _dy(terms):
    out = []
    for a, kind, mx, my, q in terms:
        if my:
            out.append((-a * my, "sin", mx, my, q) if kind == "cos" else (a * my, "cos", mx, my, q))
    return out


# --- 2D: stored k_x >= 0 modes, g = F_0 + 2 Re sum_{k >= 1} F_k e^{ikx} -------------

def _coef2d(terms, n_x, n_z):
    c = np.zeros((n_x // 2, n_z), np.complex128)
    for a, kind, mx, my, q in terms:
        assert my == 0 and mx >= 0
        zc = _cheb(q, n_z)
        if mx == 0:
            c[0] += (a if kind == "cos" else 0.0) * zc
        else:
            c[mx] += (0.5 * a if kind == "cos" else -0.5j * a) * zc
    return c


def _sum2d(c, x, z):
    out = np.zeros_like(x)
    tz = 2.0 * z - 1.0
    for k in range(c.shape[0]):
        col = C.chebval(tz, c[k].real) + 1j * C.chebval(tz, c[k].imag)
        w = 1.0 if k == 0 else 2.0
        out += w * np.real(col * np.exp(1j * k * x))
    return out


STATE_2D = {
    "u": [(1.0, "cos", 1, 0, [0, 0, 1]), (0.4, "sin", 2, 0, [0, 1, -1])],
    "w": [(0.7, "sin", 2, 0, [0, 1]), (0.3, "cos", 0, 0, [1])],
    "b": [(1.3, "cos", 1, 0, [0, 0, 0, 1]), (1.0, "cos", 0, 0, [0, 1]), (0.2, "sin", 3, 0, [1, 1])],
    "bz": [(0.9, "sin", 1, 0, [0, 1]), (2.0, "cos", 0, 0, [1])],
    "uz": [(0.6, "cos", 1, 0, [1, -1]), (-0.5, "cos", 2, 0, [0, 0, 1])],
    "wz": [(1.1, "cos", 2, 0, [0, 0, 1]), (0.5, "cos", 0, 0, [0, 1])],
    "p": [(0.8, "cos", 1, 0, [1, 0, 1])],
}


def test_rb2d_advective_terms_closed_form():
    n_x, n_z = 16, 12
    sysr = rb.RB2D(n_x, n_z, 1e6, L_x=TWO_PI)
    X = np.zeros((sysr.S, sysr.P, n_z), np.complex128)
    for name, terms in STATE_2D.items():
        X[sysr.var[name]] = _coef2d(terms, n_x, n_z)
    F = sysr.nonlinear(X)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, TWO_PI, 200)
    z = rng.uniform(0, 1, 200)
    y = np.zeros_like(x)
    S = {k: _eval(v, x, y, z) for k, v in STATE_2D.items()}
    dxS = {k: _eval(_dx(STATE_2D[k]), x, y, z) for k in ("b", "u", "w")}
    expect = {f: -(S["u"] * dxS[f] + S["w"] * S[f + "z"]) for f in ("b", "u", "w")}
    assert set(F) == {"b", "u", "w"}
    for f in ("b", "u", "w"):
        got = _sum2d(F[f], x, z)
        scale = np.abs(expect[f]).max()
        assert scale > 0.1
        assert np.abs(got - expect[f]).max() < 1e-13 * scale, f


def test_rb2d_pin_detects_a_swapped_term():
    """The closed form separates the pairings: w*uz in F_w (instead of w*wz)
    or a flipped sign gives an O(1) difference."""
    x = np.linspace(0.1, 6.0, 50)
    z = np.linspace(0.05, 0.95, 50)
    y = np.zeros_like(x)
    S = {k: _eval(v, x, y, z) for k, v in STATE_2D.items()}
    wx = _eval(_dx(STATE_2D["w"]), x, y, z)
    right = -(S["u"] * wx + S["w"] * S["wz"])
    swapped = -(S["u"] * wx + S["w"] * S["uz"])
    flipped = -(S["u"] * wx - S["w"] * S["wz"])
    assert np.abs(right - swapped).max() > 0.1
    assert np.abs(right - flipped).max() > 0.1


# --- 3D: pencil p = i_y K + i_x, complex y axis in FFT order --------------------------

def _coef3d(terms, n_x, n_y, n_z):
    K = n_x // 2
    c = np.zeros((n_y, K, n_z), np.complex128)
    slot = lambda m: m % n_y
    for a, kind, mx, my, q in terms:
        assert mx >= 0 and abs(my) < n_y // 2
        zc = _cheb(q, n_z)
        if mx == 0:
            # cos = (e^{i th} + e^{-i th}) / 2, sin = (e^{i th} - e^{-i th}) / (2i), both y slots stored
            if my == 0:
                c[0, 0] += (a if kind == "cos" else 0.0) * zc
            else:
                hp, hm = (0.5 * a, 0.5 * a) if kind == "cos" else (-0.5j * a, 0.5j * a)
                c[slot(my), 0] += hp * zc
                c[slot(-my), 0] += hm * zc
        else:
            c[slot(my), mx] += (0.5 * a if kind == "cos" else -0.5j * a) * zc
    return c.reshape(n_y * K, n_z)


def _sum3d(c, n_x, n_y, x, y, z):
    K = n_x // 2
    c3 = c.reshape(n_y, K, -1)
    tz = 2.0 * z - 1.0
    out = np.zeros_like(x)
    for iy in range(n_y):
        ky = iy if iy < n_y // 2 else iy - n_y
        for ix in range(K):
            col = C.chebval(tz, c3[iy, ix].real) + 1j * C.chebval(tz, c3[iy, ix].imag)
            w = 1.0 if ix == 0 else 2.0
            out += w * np.real(col * np.exp(1j * (ix * x + ky * y)))
    return out


STATE_3D = {
    "u": [(1.0, "cos", 1, 1, [0, 0, 1]), (0.4, "sin", 0, 2, [0, 1, -1])],
    "v": [(0.8, "sin", 1, -1, [0, 1]), (0.35, "cos", 2, 0, [1, 0, 1])],
    "w": [(0.7, "sin", 2, 1, [0, 1]), (0.3, "cos", 0, 0, [1])],
    "b": [(1.3, "cos", 1, 0, [0, 0, 0, 1]), (1.0, "cos", 0, 0, [0, 1]), (0.2, "sin", 0, 1, [1, 1])],
    "bz": [(0.9, "sin", 1, 1, [0, 1]), (2.0, "cos", 0, 0, [1])],
    "uz": [(0.6, "cos", 1, 0, [1, -1]), (-0.5, "cos", 0, 1, [0, 0, 1])],
    "vz": [(0.45, "sin", 2, -1, [1, 1]), (0.25, "cos", 0, 2, [0, 1])],
    "wz": [(1.1, "cos", 2, 0, [0, 0, 1]), (0.5, "cos", 0, 0, [0, 1])],
    "p": [(0.8, "cos", 1, 0, [1, 0, 1])],
}


def test_rb3d_advective_terms_closed_form():
    n_x, n_y, n_z = 12, 12, 10
    sysr = rb3d.RB3D(n_x, n_y, n_z, 1e6, L_x=TWO_PI, L_y=TWO_PI)
    X = np.zeros((sysr.S, sysr.P, n_z), np.complex128)
    for name, terms in STATE_3D.items():
        X[sysr.var[name]] = _coef3d(terms, n_x, n_y, n_z)
    F = sysr.nonlinear(X)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, TWO_PI, 120)
    y = rng.uniform(0, TWO_PI, 120)
    z = rng.uniform(0, 1, 120)
    S = {k: _eval(v, x, y, z) for k, v in STATE_3D.items()}
    assert set(F) == {"b", "u", "v", "w"}
    for f in ("b", "u", "v", "w"):
        fx = _eval(_dx(STATE_3D[f]), x, y, z)
        fy = _eval(_dy(STATE_3D[f]), x, y, z)
        expect = -(S["u"] * fx + S["v"] * fy + S["w"] * S[f + "z"])
        got = _sum3d(F[f], n_x, n_y, x, y, z)
        scale = np.abs(expect).max()
        assert scale > 0.1
        assert np.abs(got - expect).max() < 1e-13 * scale, f


def test_manufactured_states_are_resolved():
    """The state's coefficient arrays reproduce the closed forms (so the pin
    compares like with like): every term sits inside the stored modes."""
    rng = np.random.default_rng(2)
    x, y, z = rng.uniform(0, TWO_PI, 40), rng.uniform(0, TWO_PI, 40), rng.uniform(0, 1, 40)
    for name, terms in STATE_2D.items():
        c = _coef2d(terms, 16, 12)
        assert np.abs(_sum2d(c, x, z) - _eval(terms, x, 0 * x, z)).max() < 1e-13
    for name, terms in STATE_3D.items():
        c = _coef3d(terms, 12, 12, 10)
        assert np.abs(_sum3d(c, 12, 12, x, y, z) - _eval(terms, x, y, z)).max() < 1e-13
