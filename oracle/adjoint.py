"""Discrete adjoint of the RK222 Rayleigh-Benard step (oracle; test infrastructure).

The paper computes no gradients; this is the reference for the adjoint of
the step that the GPU path differentiates.  The state is the complex array
X[var, p, n] of T coefficients, viewed as a real vector of (Re, Im) parts
with the Euclidean inner product <A, B> = Re sum conj(A) B.  Every map of the
step is real-linear or bilinear, and its adjoint under that inner product
is written out here one operator at a time:

* complex-linear maps with matrix A (pencil solves, M, L, T-to-U conversion,
  Chebyshev transforms, dense derivative): adjoint = conjugate transpose;
* Fourier backward (k >= 0 amplitudes -> real grid values,
  g = Re f_0 + 2 sum_{k>=1} Re(f_k e^{ikx})): adjoint f_k = 2 sum_i g_i e^{-ikx_i}
  for k >= 1 and f_0 = sum_i g_i (real);
* Fourier forward (f_k = (1/N) sum_i g_i e^{-ikx_i}, k < K): adjoint
  g_i = (1/N) sum_{k<K} Re(f_k e^{ikx_i});
* multiplication by i k_x: adjoint multiplication by -i k_x;
* products F = c g_a g_b: adjoint ga_bar += c g_b F_bar, gb_bar += c g_a F_bar.

One RK222 step (Sec. "Runge-Kutta IMEX integrators", stage equations with
A = M + gamma dt L):
    A x1 = M x0 + dt gamma F(X0) + dt gamma G
    A x2 = M x0 + dt delta F(X0) + dt (1 - delta) F(X1) - dt (1 - gamma) L x1 + dt G
(G the constant boundary values).  Its adjoint, for the incoming gradient
lam2 of x2:
    mu2  = A^-H lam2
    lam1 = dt (1 - delta) J_F(X1)^H mu2 - dt (1 - gamma) L^H mu2
    mu1  = A^-H lam1
    lam0 = M^H (mu1 + mu2) + dt J_F(X0)^H (gamma mu1 + delta mu2)

Loss (the adjoint workload): J = 1/2 sum over the scale-1 grid of
(b_final - b_target)^2; control q on the scale-1 grid enters the initial
buoyancy as b0 = 1 - z + (A xi + q) z (1 - z) with bz0 = dz b0.

Pins: ``tests/test_oracle_adjoint.py`` (dot-product identities for every
operator and for the whole step, gradient against central differences).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import bases
from .timesteppers import GAMMA, DELTA, RK222, RungeKuttaIMEX


def _fourier_backward_adj(g, n_coeff, axis):
    """Adjoint of bases.fourier_backward along ``axis``."""
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    n_grid = g.shape[-1]
    f = np.fft.fft(g, axis=-1)[..., : n_coeff // 2]       # sum_i g_i e^{-ikx_i}
    f = f.astype(np.complex128)
    f[..., 1:] *= 2.0
    f[..., 0] = f[..., 0].real
    return np.moveaxis(f, -1, axis)


def _fourier_forward_adj(f, n_grid, axis):
    """Adjoint of bases.fourier_forward along ``axis``."""
    f = np.moveaxis(np.asarray(f, dtype=np.complex128), axis, -1)
    full = np.zeros(f.shape[:-1] + (n_grid,), dtype=np.complex128)
    full[..., : f.shape[-1]] = f
    g = (np.fft.ifft(full, axis=-1) * n_grid).real / n_grid  # (1/N) sum_k Re(f_k e^{ikx})
    return np.moveaxis(g, -1, axis)


def _cheb_backward_adj(g, n_coeff, axis):
    """Adjoint of bases.chebyshev_backward: T^T (real matrix)."""
    g = np.moveaxis(np.asarray(g), axis, -1)
    T = bases.chebyshev_T_matrix(n_coeff, g.shape[-1])
    return np.moveaxis(g @ T, -1, axis)


def _cheb_forward_adj(c, n_grid, axis):
    """Adjoint of bases.chebyshev_forward: T W with W = diag((2 - delta_n0)/N_g)."""
    c = np.moveaxis(np.asarray(c), axis, -1)
    n_coeff = c.shape[-1]
    w = np.full(n_coeff, 2.0 / n_grid)
    w[0] = 1.0 / n_grid
    T = bases.chebyshev_T_matrix(n_coeff, n_grid)
    return np.moveaxis((c * w) @ T.T, -1, axis)


class RBAdjoint:
    """Adjoint of RK222 steps of an oracle.rb.RB2D system."""

    def __init__(self, sysr):
        self.s = sysr
        self.rk = RungeKuttaIMEX(sysr, RK222)

    # -- grid maps ---------------------------------------------------------------
    def to_grid_adj(self, g, n_gx=None, n_gz=None):
        """Adjoint of RB2D.to_grid (g[z, x] -> c[p, n])."""
        s = self.s
        gx = _fourier_backward_adj(np.asarray(g).T, s.Nx, axis=0)      # [p, zg]
        return _cheb_backward_adj(gx, s.Nz, axis=1)

    def to_coeff_adj(self, c, n_gx, n_gz):
        """Adjoint of RB2D.to_coeff (grid n_gz x n_gx -> c[p, n])."""
        cz = _cheb_forward_adj(np.asarray(c).T, n_gz, axis=0)          # [zg, p]
        return _fourier_forward_adj(cz, n_gx, axis=1)                  # [zg, xg]

    # -- linearised nonlinear term ----------------------------------------------------
    def grid_fields(self, X):
        s, v = self.s, self.s.var
        g = lambda c: s.to_grid(c)
        return dict(u=g(X[v["u"]]), w=g(X[v["w"]]), bx=g(s.dx(X[v["b"]])), bz=g(X[v["bz"]]),
                    ux=g(s.dx(X[v["u"]])), uz=g(X[v["uz"]]), wx=g(s.dx(X[v["w"]])), wz=g(X[v["wz"]]))

    def nonlinear_adj(self, X, Fbar):
        """J_N(X)^H applied to per-equation T-coefficient adjoints Fbar[e][p, n]."""
        s, v = self.s, self.s.var
        G = self.grid_fields(X)
        gb = {e: self.to_coeff_adj(Fbar[e], s.Ngx, s.Ngz) for e in Fbar}   # grid adjoints
        bar = {k: np.zeros_like(G[k]) for k in G}
        # F_b = -(u bx + w bz), F_u = -(u ux + w uz), F_w = -(u wx + w wz)
        for e, (gx, gz) in (("b", ("bx", "bz")), ("u", ("ux", "uz")), ("w", ("wx", "wz"))):
            if e not in gb:
                continue
            r = gb[e]
            bar["u"] -= G[gx] * r
            bar[gx] -= G["u"] * r
            bar["w"] -= G[gz] * r
            bar[gz] -= G["w"] * r
        Xbar = np.zeros((s.S, s.P, s.Nz), dtype=np.complex128)
        ikx = 1j * s.kx[:, None]
        Xbar[v["u"]] += self.to_grid_adj(bar["u"])
        Xbar[v["w"]] += self.to_grid_adj(bar["w"])
        Xbar[v["bz"]] += self.to_grid_adj(bar["bz"])
        Xbar[v["uz"]] += self.to_grid_adj(bar["uz"])
        Xbar[v["wz"]] += self.to_grid_adj(bar["wz"])
        Xbar[v["b"]] += np.conj(ikx) * self.to_grid_adj(bar["bx"])
        Xbar[v["u"]] += np.conj(ikx) * self.to_grid_adj(bar["ux"])
        Xbar[v["w"]] += np.conj(ikx) * self.to_grid_adj(bar["wx"])
        return Xbar

    def rhs_adj(self, X, vbar):
        """J_{F~}(X)^H: pencil-vector adjoints vbar[p] -> state adjoint."""
        s = self.s
        N = s.Nz
        PL = bases.cheb_P_L(N)
        Fbar = {}
        eq_rows = {}
        r = 0
        for eq in s.problem.equations:
            nr = s.problem.equation_row_count(eq)
            eq_rows[eq["name"]] = (r, nr, eq["differential"])
            r += nr
        for e in ("b", "u", "w"):
            r0, nr, diff = eq_rows[e]
            out = np.zeros((s.P, N), dtype=np.complex128)
            for p in range(s.P):
                u = vbar[p][r0:r0 + nr]
                out[p] = PL[:nr, :].T @ u if diff else u
            Fbar[e] = out
        return self.nonlinear_adj(X, Fbar)

    # -- pencil algebra -------------------------------------------------------------
    def _lu(self, dt):
        return self.rk.factors.get(1.0, dt * GAMMA)

    def _solve_H(self, lu, p, rhs):
        kind, f = lu.factors[p]
        if kind == "dense":
            return sla.lu_solve(f, rhs, trans=2)
        return f.solve(rhs, trans="H")

    def step_adjoint(self, X0, X1, lam2, dt):
        """Given X0, the stage-1 state X1 and lam2 = dJ/dX2, return dJ/dX0."""
        s = self.s
        mats = s.matrices()
        lu = self._lu(dt)
        P = s.P
        l2 = [s.to_pencil(lam2, p) for p in range(P)]
        mu2 = [self._solve_H(lu, p, l2[p]) for p in range(P)]
        jf1 = self.rhs_adj(X1, [dt * (1 - DELTA) * m for m in mu2])
        lam1 = [s.to_pencil(jf1, p) - dt * (1 - GAMMA) * (mats[p][1].conj().T @ mu2[p]) for p in range(P)]
        mu1 = [self._solve_H(lu, p, lam1[p]) for p in range(P)]
        jf0 = self.rhs_adj(X0, [dt * (GAMMA * m1 + DELTA * m2) for m1, m2 in zip(mu1, mu2)])
        lam0 = [mats[p][0].conj().T @ (mu1[p] + mu2[p]) + s.to_pencil(jf0, p) for p in range(P)]
        return s.from_pencils(lam0)

    def stage1(self, X0, dt):
        """The stage-1 state of a step from X0 (for the adjoint)."""
        s = self.s
        mats = s.matrices()
        lu = self._lu(dt)
        F0 = s.rhs_vectors(X0)
        return s.from_pencils([lu.solve(p, mats[p][0] @ s.to_pencil(X0, p) + dt * GAMMA * F0[p])
                               for p in range(s.P)])

    # -- the control-to-loss map ---------------------------------------------------------
    def initial_state_q(self, noise, q, amplitude=1e-3):
        s = self.s
        z = bases.chebyshev_grid(s.Nz)[:, None]
        b_grid = 1.0 - z + (amplitude * noise + q) * z * (1.0 - z)
        cb = s.to_coeff(b_grid)                                      # scale-1 forward
        X = np.zeros((s.S, s.P, s.Nz), dtype=np.complex128)
        X[s.var["b"]] = cb
        X[s.var["bz"]] = bases.chebyshev_derivative(cb, 0.0, 1.0, axis=1)
        return X

    def initial_state_adj(self, Xbar):
        """d(loss)/dq from the adjoint of the initial state."""
        s = self.s
        D = bases.cheb_D_TT(s.Nz) * 2.0
        cbar = Xbar[s.var["b"]] + Xbar[s.var["bz"]] @ D.conj()       # (D c)^H adjoint: c_bar += D^T bz_bar
        cz = _cheb_forward_adj(cbar.T, s.Nz, axis=0)                   # [z, p]
        g = _fourier_forward_adj(cz, s.Nx, axis=1)                     # [z, x]
        z = bases.chebyshev_grid(s.Nz)[:, None]
        return g * z * (1.0 - z)

    def loss_and_grad(self, noise, target_grid, q, dt, nsteps):
        s = self.s
        X = self.initial_state_q(noise, q)
        traj = []
        for _ in range(nsteps):
            X1 = self.stage1(X, dt)
            traj.append((X, X1))
            X = self.rk.step(X, dt)
        b = s.to_grid(X[s.var["b"]], s.Nx, s.Nz)
        r = b - target_grid
        J = 0.5 * float(np.sum(r * r))
        lam = np.zeros_like(X)
        lam[s.var["b"]] = self.to_grid_adj_scale1(r)
        for (X0, X1) in reversed(traj):
            lam = self.step_adjoint(X0, X1, lam, dt)
        return J, self.initial_state_adj(lam)

    def to_grid_adj_scale1(self, g):
        """Adjoint of to_grid(c, N_x, N_z) (scale-1 grid)."""
        s = self.s
        gx = _fourier_backward_adj(np.asarray(g).T, s.Nx, axis=0)
        return _cheb_backward_adj(gx, s.Nz, axis=1)
