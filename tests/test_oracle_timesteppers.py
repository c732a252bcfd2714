"""Pins for oracle.timesteppers on linear problems with closed-form solutions.

* a z-independent diffusion mode cos(k x) under Neumann walls is a T_0-only
  polynomial, so the tau discretisation is exact and the step must multiply
  it by the scheme's amplification factor, to rounding:
  RK222 (ARS(2,2,2)): R(h) = (1 + (2 gamma - 1) h) / (1 + gamma h)^2,
  SBDF1 then SBDF2: x_1 = x_0 / (1 + h), (3/2 + h) x_{n+1} = 2 x_n - x_{n-1} / 2;
* a Dirichlet mode sin(pi z) cos(k x) decays at lambda = kappa (k^2 + pi^2)
  to spectral accuracy, and the time error is second order;
* the tau polynomial U_{N-1} has zero integral for even N, so the Neumann
  diffusion step conserves the mean exactly (Sec. "Integration").
"""
import numpy as np
import pytest

from oracle import bases
from oracle.problem import TauProblem, LinearPencilSystem
from oracle import timesteppers as ts

KAPPA = 0.05
L_X = 4.0


def diffusion(N, bc="neumann"):
    pr = TauProblem(["c", "cz"], N, 0.0, 1.0)
    pr.add_equation("cz_def", L_terms=[("c", "dz", 1.0), ("cz", "I", -1.0)])
    pr.add_equation("c", M_terms=[("c", "I", 1.0)],
                    L_terms=[("c", "I", lambda k: KAPPA * k * k), ("cz", "dz", -KAPPA)])
    v = "cz" if bc == "neumann" else "c"
    pr.add_bc(v, "left", value=0.0)
    pr.add_bc(v, "right", value=0.0)
    return pr


def _mode_state(sysm, N, n_kx, zfun, dzfun):
    z = bases.chebyshev_grid(N)
    X = np.zeros((2, sysm.P, N), complex)
    X[0, n_kx] = 0.5 * bases.chebyshev_forward(zfun(z), N)    # cos(k x) -> 1/2 e^{ikx}
    X[1, n_kx] = 0.5 * bases.chebyshev_forward(dzfun(z), N)
    return X


def R_rk222(h):
    g = ts.GAMMA
    return (1 + (2 * g - 1) * h) / (1 + g * h) ** 2


def test_ars222_tableau_order_conditions():
    H, A, c = ts.RK222["H"], ts.RK222["A"], ts.RK222["c"]
    b = H[-1]                                   # stiffly accurate: weights = last row
    assert np.allclose(A[-1, :-1].sum(), 1.0) and np.allclose(b.sum(), 1.0)
    assert np.allclose(b @ c, 0.5)             # second-order condition (implicit)
    assert np.allclose(A[-1] @ c, 0.5)         # second-order condition (explicit)
    assert np.allclose(H.sum(axis=1), c) and np.allclose(A.sum(axis=1), c)


@pytest.mark.parametrize("N", [8, 16])
def test_rk222_neumann_mode_exact_amplification(N):
    kx = 2 * np.pi * np.arange(4) / L_X
    sysm = LinearPencilSystem(diffusion(N), kx)
    X = _mode_state(sysm, N, 3, np.ones_like, np.zeros_like)
    stepper = ts.RungeKuttaIMEX(sysm)
    dt = 0.3
    amp0 = X[0, 3, 0]
    for n in range(1, 8):
        X = stepper.step(X, dt)
        h = KAPPA * kx[3] ** 2 * dt
        assert abs(X[0, 3, 0] - amp0 * R_rk222(h) ** n) < 1e-14
        assert np.abs(X[0, 3, 1:]).max() < 1e-14 and np.abs(X[1]).max() < 1e-13


def test_sbdf2_neumann_mode_recurrence():
    N = 12
    kx = 2 * np.pi * np.arange(3) / L_X
    sysm = LinearPencilSystem(diffusion(N), kx)
    X = _mode_state(sysm, N, 2, np.ones_like, np.zeros_like)
    stepper = ts.SBDF(sysm, order=2)
    dt = 0.2
    h = KAPPA * kx[2] ** 2 * dt
    seq = [X[0, 2, 0]]
    seq.append(seq[0] / (1 + h))
    for n in range(6):
        seq.append((2 * seq[-1] - 0.5 * seq[-2]) / (1.5 + h))
    for n in range(1, 8):
        X = stepper.step(X, dt)
        assert abs(X[0, 2, 0] - seq[n]) < 1e-14


def test_dirichlet_mode_spectral_accuracy_and_second_order():
    N = 32
    kx = 2 * np.pi * np.arange(3) / L_X
    sysm = LinearPencilSystem(diffusion(N, "dirichlet"), kx)
    lam = KAPPA * (kx[1] ** 2 + np.pi ** 2)
    T = 1.0
    errs = {}
    for name, make in [("rk", lambda: ts.RungeKuttaIMEX(sysm)), ("sbdf", lambda: ts.SBDF(sysm, 2))]:
        errs[name] = []
        for nsteps in (20, 40, 80):
            dt = T / nsteps
            X = _mode_state(sysm, N, 1, lambda z: np.sin(np.pi * z), lambda z: np.pi * np.cos(np.pi * z))
            a0 = X[0, 1].copy()
            st = make()
            for _ in range(nsteps):
                X = st.step(X, dt)
            if name == "rk":
                # spectral accuracy: time-discrete amplification of the exact mode
                assert np.abs(X[0, 1] - a0 * R_rk222(lam * dt) ** nsteps).max() < 1e-12
            errs[name].append(np.abs(X[0, 1] - a0 * np.exp(-lam * T)).max())
        r = np.array(errs[name][:-1]) / np.array(errs[name][1:])
        assert np.all((r > 3.6) & (r < 4.4)), (name, r)


def test_neumann_diffusion_conserves_mean_even_N():
    N = 16
    sysm = LinearPencilSystem(diffusion(N), np.array([0.0]))
    z = bases.chebyshev_grid(N)
    X = np.zeros((2, 1, N), complex)
    X[0, 0] = bases.chebyshev_forward(2 + np.cos(np.pi * z) + 0.3 * np.cos(2 * np.pi * z), N)
    X[1, 0] = bases.chebyshev_forward(-np.pi * np.sin(np.pi * z) - 0.6 * np.pi * np.sin(2 * np.pi * z), N)
    integ = bases.cheb_integrate_vector(N) * 0.5          # int_0^1 dz
    m0 = integ @ X[0, 0]
    st = ts.RungeKuttaIMEX(sysm)
    for _ in range(20):
        X = st.step(X, 0.05)
    assert abs(integ @ X[0, 0] - m0) < 1e-14
    assert abs(m0 - 2.0) < 1e-11          # truncation of cos(pi z) at N = 16


# ---------------------------------------------------------------------------
# RK443 (ARS(4,4,3))


def test_ars443_tableau_third_order_conditions():
    """Third-order conditions of the implicit and explicit tableaux and of
    their coupling (additive Runge-Kutta), with the weights the last rows
    (X^{n+1} = X^s)."""
    H, A, c = ts.RK443["H"], ts.RK443["A"], ts.RK443["c"]
    assert np.allclose(H.sum(axis=1), c) and np.allclose(A.sum(axis=1), c)
    assert np.all(np.triu(A) == 0) and np.all(np.triu(H, 1) == 0)
    assert np.allclose(np.diag(H)[1:], 0.5)            # one factor for every stage
    for b in (H[-1], A[-1]):
        assert np.isclose(b.sum(), 1.0)
        assert np.isclose(b @ c, 1 / 2)
        assert np.isclose(b @ (c * c), 1 / 3)
        assert np.isclose(b @ (A @ c), 1 / 6) and np.isclose(b @ (H @ c), 1 / 6)


def test_rk443_dirichlet_mode_third_order():
    N = 32
    kx = 2 * np.pi * np.arange(3) / L_X
    sysm = LinearPencilSystem(diffusion(N, "dirichlet"), kx)
    lam = KAPPA * (kx[1] ** 2 + np.pi ** 2)
    T = 1.0
    errs = []
    for nsteps in (5, 10, 20):
        dt = T / nsteps
        X = _mode_state(sysm, N, 1, lambda z: np.sin(np.pi * z), lambda z: np.pi * np.cos(np.pi * z))
        a0 = X[0, 1].copy()
        st = ts.RungeKuttaIMEX(sysm, ts.RK443)
        for _ in range(nsteps):
            X = st.step(X, dt)
        errs.append(np.abs(X[0, 1] - a0 * np.exp(-lam * T)).max())
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 7.0) & (r < 9.0)), r


class _Scalar:
    """x' = -lam x - x^2 as a one-pencil system: M = 1, L = lam, F = -x^2."""

    def __init__(self, lam):
        import scipy.sparse as sps
        self.P = 1
        self._m = [(sps.csr_matrix(np.array([[1.0]])), sps.csr_matrix(np.array([[lam]])))]

    def matrices(self):
        return self._m

    def rhs_vectors(self, X):
        return [-X * X]

    def to_pencil(self, X, p):
        return X

    def from_pencils(self, vecs):
        return vecs[0]


@pytest.mark.parametrize("name,order", [("RK222", 2), ("RK443", 3)])
def test_imex_order_on_stiff_linear_quadratic_scalar(name, order):
    """Both parts of the scheme at once: x(t) = lam x0 e^{-lam t} / (lam +
    x0 (1 - e^{-lam t})) solves x' = -lam x - x^2."""
    lam, x0, T = 2.0, 1.0, 1.0
    exact = lam * x0 * np.exp(-lam * T) / (lam + x0 * (1 - np.exp(-lam * T)))
    errs = []
    for nsteps in (10, 20, 40):
        st = ts.RungeKuttaIMEX(_Scalar(lam), getattr(ts, name))
        X = np.array([x0])
        for _ in range(nsteps):
            X = st.step(X, T / nsteps)
        errs.append(abs(X[0] - exact))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(np.log2(r) - order) < 0.3), r


# ---------------------------------------------------------------------------
# SBDF3 / SBDF4


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_sbdf_coefficients_are_consistent(order):
    """sum a_j = 0 and sum_j j a_j = -1 (exact for constants and lines,
    with a in units of 1/dt), sum c_j = 1 (extrapolation of constants)."""
    a, b, c = ts.SBDF.coefficients(order, 1.0)
    j = np.arange(order + 1)
    assert abs(a.sum()) < 1e-14 and abs((j * a).sum() + 1.0) < 1e-14
    assert abs(c.sum() - 1.0) < 1e-14 and b[0] == 1.0 and np.all(b[1:] == 0)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_sbdf_order_from_exact_history(order):
    """x' = -lam x - x^2 with the exact solution as the start-up history:
    the global error falls at the scheme's order (a lower-order start would
    mask it)."""
    lam, x0, T = 2.0, 1.0, 1.0

    def exact(t):
        return lam * x0 * np.exp(-lam * t) / (lam + x0 * (1 - np.exp(-lam * t)))

    errs = []
    for nsteps in (80, 160, 320):
        dt = T / nsteps
        sysm = _Scalar(lam)
        st = ts.SBDF(sysm, order)
        M, L = sysm.matrices()[0]
        for k in range(order - 1, 0, -1):          # oldest first: the list is newest-first
            xk = np.array([exact(-k * dt)])
            st.hist_MX.insert(0, [M @ xk])
            st.hist_LX.insert(0, [L @ xk])
            st.hist_F.insert(0, sysm.rhs_vectors(xk))
        st.iteration = order - 1
        X = np.array([x0])
        for _ in range(nsteps):
            X = st.step(X, dt)
        errs.append(abs(X[0] - exact(T)))
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(np.log2(r) - order) < 0.35), r


# ---------------------------------------------------------------------------
# CNAB1 / CNAB2


@pytest.mark.parametrize("order", [1, 2])
def test_cnab_coefficients_are_consistent(order):
    """Trapezoidal implicit part (b = (1/2, 1/2)), first-difference a, and
    Adams-Bashforth weights: sum c_j = 1, and for CNAB2 sum_j c_j (1 - j) =
    1/2 (the extrapolation to the midpoint t^{n-1/2} is exact for lines)."""
    a, b, c = ts.CNAB.coefficients(order, 1.0)
    assert abs(a.sum()) < 1e-15 and a[0] == 1.0
    assert b[0] == 0.5 and b[1] == 0.5 and abs(b.sum() - 1.0) < 1e-15
    assert abs(c.sum() - 1.0) < 1e-15
    if order == 2:
        j = np.arange(order + 1)
        assert abs((c * (1 - j)).sum() - 0.5) < 1e-15


def test_cnab_neumann_mode_crank_nicolson_factor():
    """F = 0: both orders reduce to the trapezoidal rule, x_{n+1} =
    x_n (1 - h/2) / (1 + h/2) for the z-independent diffusion mode."""
    N = 12
    kx = 2 * np.pi * np.arange(3) / L_X
    sysm = LinearPencilSystem(diffusion(N), kx)
    X = _mode_state(sysm, N, 2, np.ones_like, np.zeros_like)
    stepper = ts.CNAB(sysm, order=2)
    dt = 0.2
    h = KAPPA * kx[2] ** 2 * dt
    amp0 = X[0, 2, 0]
    for n in range(1, 8):
        X = stepper.step(X, dt)
        assert abs(X[0, 2, 0] - amp0 * ((1 - h / 2) / (1 + h / 2)) ** n) < 1e-14
        assert np.abs(X[0, 2, 1:]).max() < 1e-14


def test_cnab2_second_order():
    """x' = -lam x - x^2 (closed form): second order from the CNAB1 start and
    from an exact start-up history."""
    lam, x0, T = 2.0, 1.0, 1.0

    def exact(t):
        return lam * x0 * np.exp(-lam * t) / (lam + x0 * (1 - np.exp(-lam * t)))

    for warm in (False, True):
        errs = []
        for nsteps in (80, 160, 320):
            dt = T / nsteps
            sysm = _Scalar(lam)
            st = ts.CNAB(sysm, 2)
            if warm:
                M, L = sysm.matrices()[0]
                xk = np.array([exact(-dt)])
                st.hist_MX.insert(0, [M @ xk])
                st.hist_LX.insert(0, [L @ xk])
                st.hist_F.insert(0, sysm.rhs_vectors(xk))
                st.iteration = 1
            X = np.array([x0])
            for _ in range(nsteps):
                X = st.step(X, dt)
            errs.append(abs(X[0] - exact(T)))
        r = np.array(errs[:-1]) / np.array(errs[1:])
        assert np.all(np.abs(np.log2(r) - 2) < 0.3), (warm, r)
