"""Pins for oracle.rb3d: the 3D Rayleigh-Benard system.

* the complex y transform reproduces single modes exactly and round-trips
  band-limited data (closed forms of the discrete Fourier sums);
* a y-independent state with v = 0 evolves exactly as the 2D system
  (oracle.rb), whose pencils and products are pinned separately;
* the linear growth rate depends on (k_x, k_y) only through |k| (rotation
  invariance), and an oblique wave at |k| = k_c is marginal at the textbook
  Ra_c (tests/golden/rb_onset.txt);
* the conductive state is an exact steady state of the nonlinear step;
* the rounding-floor variants (DCT transforms with numpy's derivative
  recurrence, dense LAPACK or natural-order SuperLU for the pencils) step a
  random state to the default's result up to rounding, so they compute the
  same thing.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bases, rb, rb3d
from oracle import timesteppers as ts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rb_onset.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def test_y_transform_single_modes_and_round_trip():
    Ny, Ly = 8, 4.0
    y = bases.fourier_grid(12, Ly)
    n = 3
    g = np.exp(2j * np.pi * n * y / Ly) + 0.5 * np.exp(-2j * np.pi * 2 * y / Ly)
    f = bases.fourier_c_forward(g, Ny)
    ref = np.zeros(Ny, complex)
    ref[3], ref[Ny - 2] = 1.0, 0.5
    assert np.abs(f - ref).max() < 1e-15
    back = bases.fourier_c_backward(f, 12)
    assert np.abs(back - g).max() < 1e-14
    # the Nyquist slot is dropped on the way in and ignored on the way out
    f2 = f.copy()
    f2[Ny // 2] = 7.0
    assert np.abs(bases.fourier_c_backward(f2, 12) - g).max() < 1e-14
    assert bases.fourier_c_forward(np.cos(np.pi * Ny * y / Ly), Ny)[Ny // 2] == 0


def test_grid_round_trip():
    s = rb3d.RB3D(8, 8, 8, 1e5)
    rng = np.random.default_rng(0)
    g = rng.standard_normal((8, 8, 8))
    c = s.to_coeff(g)
    c2 = s.to_coeff(s.to_grid(c))
    assert np.abs(c2 - c).max() < 1e-14 * np.abs(c).max()
    # real data: the k_x = 0 column is Hermitian in k_y
    c3 = c.reshape(8, 4, 8)
    iy = np.arange(8)
    assert np.abs(c3[(-iy) % 8, 0] - np.conj(c3[iy, 0])).max() < 1e-15


@pytest.mark.parametrize("scheme", ["RK222", "SBDF2"])
def test_y_independent_state_reduces_to_2d(scheme):
    Nx, Ny, Nz, Ra, dt = 16, 8, 16, 1e6, 1e-3
    s3 = rb3d.RB3D(Nx, Ny, Nz, Ra)
    s2 = rb.RB2D(Nx, Nz, Ra)
    xi = np.random.default_rng(3).standard_normal((Nz, Nx))
    X2 = s2.initial_state(xi * 100)
    X2[s2.var["u"]] = 1e-2 * s2.to_coeff(np.sin(2 * np.pi * bases.fourier_grid(Nx, 4.0))[None, :]
                                          * np.ones((Nz, 1)))
    X3 = np.zeros((s3.S, s3.P, Nz), complex)
    for v in rb.RB_VARIABLES:
        X3[s3.var[v], : s3.K] = X2[s2.var[v]]              # the k_y = 0 pencils
    mk = (lambda sysr: ts.RungeKuttaIMEX(sysr)) if scheme == "RK222" else (lambda sysr: ts.SBDF(sysr, 2))
    st2, st3 = mk(s2), mk(s3)
    for _ in range(3):
        X2, X3 = st2.step(X2, dt), st3.step(X3, dt)
    for v in rb.RB_VARIABLES:
        assert np.abs(X3[s3.var[v], : s3.K] - X2[s2.var[v]]).max() < 1e-12, v
    assert np.abs(X3[:, s3.K:]).max() < 1e-14             # no k_y != 0 content appears
    assert np.abs(X3[s3.var["v"]]).max() < 1e-14 and np.abs(X3[s3.var["vz"]]).max() < 1e-14


def _max_growth(Ra, k, N=24):
    M, L = rb3d.rb3d_onset_pencil(N, Ra, 1.0, k)
    w = sla.eig(-L.toarray(), M.toarray(), right=False)
    return np.max(w[np.isfinite(w)].real)


def test_growth_rate_rotation_invariance_and_onset():
    g = _golden()
    Ra_c, k_c = g["Ra_c"], g["k_c"]
    k = 2.7
    ref = _max_growth(3000.0, (k, 0.0))
    for th in (0.3, 1.1, np.pi / 2):
        assert abs(_max_growth(3000.0, (k * np.cos(th), k * np.sin(th))) - ref) < 1e-9
    kk = (k_c * np.cos(0.7), k_c * np.sin(0.7))
    assert _max_growth(0.99 * Ra_c, kk) < 0 < _max_growth(1.01 * Ra_c, kk)


def test_conductive_state_is_steady():
    s = rb3d.RB3D(8, 8, 12, 1e6)
    X0 = s.conductive_state()
    st = ts.RungeKuttaIMEX(s)
    X = X0
    for _ in range(2):
        X = st.step(X, 1e-2)
    assert np.abs(X - X0).max() < 1e-12


def test_rounding_floor_variants_agree():
    args = (8, 8, 16, 1e6)
    noise = np.random.default_rng(4).standard_normal((16, 8, 8)) * 30.0
    ref = None
    for cheb, lu in (("mmt", "auto"), ("dct", "auto"), ("mmt", "dense"), ("mmt", "natural")):
        sysr = rb3d.RB3D(*args, cheb_method=cheb, lu_method=lu)
        X = sysr.initial_state(noise)
        st = ts.RungeKuttaIMEX(sysr, ts.RK222)
        for _ in range(2):
            X = st.step(X, 1e-3)
        if ref is None:
            ref = X
            continue
        for i, v in enumerate(rb3d.RB3D_VARIABLES):
            nr = np.linalg.norm(ref[i])
            err = np.linalg.norm(X[i] - ref[i]) / max(nr, 1e-300)
            assert err < 1e-9 or np.linalg.norm(X[i] - ref[i]) < 1e-14, (cheb, lu, v, err)

