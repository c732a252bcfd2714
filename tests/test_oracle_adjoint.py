"""Pins for oracle.adjoint: every adjoint operator against the dot-product
identity <A x, y> = <x, A^H y> (real inner product Re sum conj(a) b), the
adjoint of a whole RK222 step against central differences of the step, and
the gradient of the loss against central differences (relative 1e-6)."""
import numpy as np
import pytest

from oracle import rb as orb
from oracle.adjoint import RBAdjoint
import seeded_inputs as si

RNG = np.random.default_rng(77)


def ip(a, b):
    return float(np.real(np.sum(np.conj(a) * b)))


def _rand_state(s, scale=1.0):
    X = scale * (RNG.standard_normal((s.S, s.P, s.Nz)) + 1j * RNG.standard_normal((s.S, s.P, s.Nz)))
    return X


@pytest.fixture(scope="module")
def sysr():
    return orb.RB2D(16, 12, 1e5)


def test_grid_maps_dot_product(sysr):
    adj = RBAdjoint(sysr)
    c = _rand_state(sysr)[0]
    g = RNG.standard_normal((sysr.Ngz, sysr.Ngx))
    assert abs(ip(sysr.to_grid(c), g) - ip(c, adj.to_grid_adj(g))) < 1e-10 * abs(ip(sysr.to_grid(c), g))
    g1 = RNG.standard_normal((sysr.Nz, sysr.Nx))
    lhs = ip(sysr.to_grid(c, sysr.Nx, sysr.Nz), g1)
    assert abs(lhs - ip(c, adj.to_grid_adj_scale1(g1))) < 1e-10 * abs(lhs)
    h = RNG.standard_normal((sysr.Ngz, sysr.Ngx))
    cbar = _rand_state(sysr)[1]
    lhs = ip(sysr.to_coeff(h), cbar)
    assert abs(lhs - ip(h, adj.to_coeff_adj(cbar, sysr.Ngx, sysr.Ngz))) < 1e-10 * abs(lhs)


def test_linearised_rhs_dot_product(sysr):
    adj = RBAdjoint(sysr)
    X, dX = _rand_state(sysr), _rand_state(sysr)
    eps = 1e-3
    Fp, Fm = sysr.rhs_vectors(X + eps * dX), sysr.rhs_vectors(X - eps * dX)
    JdX = [(a - b) / (2 * eps) for a, b in zip(Fp, Fm)]          # exact: F is bilinear
    V = [RNG.standard_normal(len(v)) + 1j * RNG.standard_normal(len(v)) for v in JdX]
    lhs = sum(ip(a, b) for a, b in zip(JdX, V))
    rhs = ip(dX, adj.rhs_adj(X, V))
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)


def test_step_adjoint_against_linearised_step(sysr):
    adj = RBAdjoint(sysr)
    dt = 1e-2
    X0 = _rand_state(sysr, 0.05)
    dX = _rand_state(sysr)
    lam = _rand_state(sysr)
    eps = 1e-6
    step = lambda X: adj.rk.step(X, dt)
    JdX = (step(X0 + eps * dX) - step(X0 - eps * dX)) / (2 * eps)
    X1 = adj.stage1(X0, dt)
    g = adj.step_adjoint(X0, X1, lam, dt)
    lhs, rhs = ip(JdX, lam), ip(dX, g)
    assert abs(lhs - rhs) < 1e-7 * abs(lhs), (lhs, rhs)


def test_gradient_against_central_differences():
    s = orb.RB2D(16, 12, 1e5)
    adj = RBAdjoint(s)
    noise = si.rb_noise(5, s.Nz, s.Nx) * 50.0          # larger perturbation: nonlinear terms matter
    target = s.to_grid(adj.initial_state_q(si.rb_noise(6, s.Nz, s.Nx) * 50.0, 0.0)[0], s.Nx, s.Nz)
    q = 0.01 * RNG.standard_normal((s.Nz, s.Nx))
    dt, nsteps = 1e-2, 4
    J, grad = adj.loss_and_grad(noise, target, q, dt, nsteps)
    for trial in range(3):
        d = RNG.standard_normal((s.Nz, s.Nx))
        eps = 1e-4
        Jp, _ = adj.loss_and_grad(noise, target, q + eps * d, dt, nsteps)
        Jm, _ = adj.loss_and_grad(noise, target, q - eps * d, dt, nsteps)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * d))
        assert abs(fd - an) < 1e-6 * abs(fd), (fd, an)
