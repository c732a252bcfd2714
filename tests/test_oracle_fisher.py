"""Pins for oracle.fisher: the Fisher-KPP example of Sec. "Codebase structure".

* a spatially uniform state stays uniform (only the k_x = 0, T_0 coefficient
  is non-zero, and it satisfies the Neumann rows), so it follows the logistic
  equation u' = R u (1 - u) with only time-discretization error: second-order
  convergence of RK222 and third-order of RK443 to the closed form;
* with R = 0 the mode cos(k x) cos(pi z) (Neumann at both walls) decays at
  D (k^2 + pi^2), with second-order time error;
* the dealiased square -R u^2 equals the brute-force truncated product of the
  expansions (Fourier convolution and T_a T_b = (T_{a+b} + T_{|a-b|}) / 2).
"""
import numpy as np
import pytest

from oracle import bases
from oracle import fisher as of
from oracle import timesteppers as ts


def _run(sysm, X, tableau, dt, nsteps):
    st = ts.RungeKuttaIMEX(sysm, tableau)
    for _ in range(nsteps):
        X = st.step(X, dt)
    return X


@pytest.mark.parametrize("name,order", [("RK222", 2), ("RK443", 3)])
def test_uniform_state_follows_logistic_closed_form(name, order):
    u0, R, T = 0.2, 1.0, 1.0
    exact = u0 * np.exp(R * T) / (1 - u0 + u0 * np.exp(R * T))
    sysm = of.FisherKPP(8, 8, D=0.1, R=R)
    errs = []
    for nsteps in (16, 32, 64):
        X = sysm.initial_state(np.full((8, 8), u0))
        X = _run(sysm, X, getattr(ts, name), T / nsteps, nsteps)
        rest = X.copy()
        rest[0, 0, 0] = 0.0
        assert np.abs(rest).max() < 1e-14                 # stays uniform
        errs.append(abs(X[0, 0, 0] - exact))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(np.log2(r) - order) < 0.3), r


def test_pure_diffusion_mode_decay():
    Nx, Nz, D = 8, 24, 0.1
    sysm = of.FisherKPP(Nx, Nz, D=D, R=0.0)
    k = sysm.kx[1]
    lam = D * (k * k + np.pi ** 2)
    x = bases.fourier_grid(Nx, sysm.Lx)[None, :]
    z = bases.chebyshev_grid(Nz)[:, None]
    T, errs = 1.0, []
    for nsteps in (10, 20, 40):
        X = sysm.initial_state(np.cos(k * x) * np.cos(np.pi * z))
        a0 = X[0, 1].copy()
        X = _run(sysm, X, ts.RK222, T / nsteps, nsteps)
        assert np.abs(X[:, 0]).max() < 1e-14 and np.abs(X[:, 2:]).max() < 1e-14
        errs.append(np.abs(X[0, 1] - a0 * np.exp(-lam * T)).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 3.6) & (r < 4.4)), r


def test_dealiased_square_equals_brute_force_product():
    Nx, Nz, R = 8, 6, 0.7
    K = Nx // 2
    sysm = of.FisherKPP(Nx, Nz, D=0.1, R=R)
    rng = np.random.default_rng(5)
    c = rng.standard_normal((K, Nz)) + 1j * rng.standard_normal((K, Nz))
    c[0] = c[0].real                                      # real field: real k = 0 column
    X = np.zeros((2, K, Nz), complex)
    X[0] = c
    got = sysm.nonlinear(X)["u"]
    # full spectrum of the real field, k = -(K-1) .. K-1 (Nyquist dropped)
    f = {k: c[k] for k in range(K)}
    f.update({-k: np.conj(c[k]) for k in range(1, K)})
    ref = np.zeros((K, Nz), complex)
    for k1, a1 in f.items():
        for k2, a2 in f.items():
            k = k1 + k2
            if not 0 <= k < K:
                continue
            for a in range(Nz):
                for b in range(Nz):
                    for m in (a + b, abs(a - b)):
                        if m < Nz:
                            ref[k, m] += 0.5 * a1[a] * a2[b]
    assert np.abs(got - (-R) * ref).max() < 1e-13 * np.abs(ref).max()
