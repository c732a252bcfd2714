"""Pins for oracle.rb: the Rayleigh-Benard pencils and nonlinear RHS.

* linear onset: the growth rate of the linearisation about the conductive
  state changes sign at the textbook Ra_c = 1707.76, k_c = 3.117 for no-slip,
  fixed-temperature walls (tests/golden/rb_onset.txt);
* the conductive state is an exact polynomial steady state of the full
  nonlinear step;
* after steps from the seeded initial state the boundary conditions, the
  divergence constraint and the first-order definitions hold;
* the initial state reproduces the grid buoyancy (less its Nyquist part).
"""
import os

import numpy as np
import scipy.linalg as sla
import pytest

from oracle import bases, rb
from oracle import timesteppers as ts
import seeded_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rb_onset.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def _max_growth(Ra, k, N=32):
    M, L = rb.rb_onset_pencil(N, Ra, 1.0, k)
    w = sla.eig(-L.toarray(), M.toarray(), right=False)
    return np.max(w[np.isfinite(w)].real)


def test_linear_onset_matches_textbook():
    g = _golden()
    Ra_c, k_c = g["Ra_c"], g["k_c"]
    assert _max_growth(0.99 * Ra_c, k_c) < 0 < _max_growth(1.01 * Ra_c, k_c)
    assert abs(_max_growth(Ra_c, k_c)) < 1e-5
    # k_c is the most unstable wavenumber at onset
    assert _max_growth(Ra_c, 0.85 * k_c) < 0 and _max_growth(Ra_c, 1.15 * k_c) < 0


@pytest.mark.parametrize("scheme", ["RK222", "SBDF2"])
def test_conductive_state_is_steady(scheme):
    sysr = rb.RB2D(16, 16, 1e6)
    X0 = sysr.conductive_state()
    st = ts.RungeKuttaIMEX(sysr) if scheme == "RK222" else ts.SBDF(sysr, 2)
    X = X0
    for _ in range(3):
        X = st.step(X, 1e-2)
    assert np.abs(X - X0).max() < 1e-12     # roundoff x O(N) derivative entries


def test_invariants_after_steps():
    sysr = rb.RB2D(32, 16, 1e6)
    X = sysr.initial_state(si.rb_noise(42, 16, 32))
    st = ts.RungeKuttaIMEX(sysr)
    for _ in range(5):
        X = st.step(X, 1e-3)
    v = sysr.var
    N = sysr.Nz
    left, right = bases.cheb_left_vector(N), bases.cheb_right_vector(N)
    b, u, w = X[v["b"]], X[v["u"]], X[v["w"]]
    assert abs(b[0] @ left - 1) < 1e-13 and abs(b[0] @ right) < 1e-13
    assert np.abs(b[1:] @ left).max() < 1e-13 and np.abs(b[1:] @ right).max() < 1e-13
    for f in (u, w):
        assert np.abs(f @ left).max() < 1e-13
    assert np.abs(u @ right).max() < 1e-13 and np.abs(w[1:] @ right).max() < 1e-13
    assert abs(X[v["p"], 0] @ right) < 1e-13                       # gauge
    div = sysr.dx(u) + X[v["wz"]]
    assert np.abs(div).max() < 1e-12
    # first-order definitions hold in the U basis except the tau row
    PL, DTU = bases.cheb_P_L(N), 2 * bases.cheb_D_TU(N)
    for a, az in (("b", "bz"), ("u", "uz"), ("w", "wz")):
        r = X[v[a]] @ DTU.T - X[v[az]] @ PL.T
        assert np.abs(r[:, : N - 1]).max() < 1e-11
    assert np.abs(u).max() > 1e-12                                 # the flow did start


def test_initial_state_reproduces_grid_buoyancy():
    Nx, Nz = 16, 12
    sysr = rb.RB2D(Nx, Nz, 1e6)
    xi = si.rb_noise(3, Nz, Nx)
    X = sysr.initial_state(xi)
    z = bases.chebyshev_grid(Nz)[:, None]
    bg = 1 - z + 1e-3 * xi * z * (1 - z)
    nyq = (bg * (-1.0) ** np.arange(Nx)).mean(axis=1, keepdims=True) * (-1.0) ** np.arange(Nx)
    back = sysr.to_grid(X[sysr.var["b"]], Nx, Nz)
    assert np.abs(back - (bg - nyq)).max() < 1e-14
    d = bases.chebyshev_backward(X[sysr.var["bz"]], Nz, axis=1)
    assert abs(d[0].real.mean() + 1.0) < 1e-3     # dz(1 - z) = -1 dominates
