"""Rayleigh-Benard convection in first-order tau form (oracle; test infrastructure).

The paper does not write these equations; this is the reading used on both
sides.  Free-fall units with
kappa = (Ra Pr)^(-1/2), nu = (Ra/Pr)^(-1/2); z in [0, 1] (Chebyshev),
x in [0, L_x) (Fourier), buoyancy b, gravity along -z.  In the paper's IVP
form  M dt(X) + L X = F(X)  (Sec. "Initial value solver", Eq. ivp) with
X = (b, p, u, w, bz, uz, wz):

    bz_def:  dz(b) - bz = 0
    uz_def:  dz(u) - uz = 0
    wz_def:  dz(w) - wz = 0
    b:       dt(b) - kappa (dx dx b + dz bz)            = -(u dx b + w bz)
    u:       dt(u) - nu (dx dx u + dz uz) + dx p        = -(u dx u + w uz)
    w:       dt(w) - nu (dx dx w + dz wz) + dz p - b    = -(u dx w + w wz)
    div:     dx u + wz = 0            (no z-derivative: algebraic, no tau row)

    b(0) = 1, b(1) = 0, u(0) = u(1) = 0, w(0) = 0,
    w(1) = 0 for k_x != 0, p(1) = 0 for k_x = 0 (gauge; the ``condition``
    mechanism of Sec. "Equation parsing").

The nonlinear terms are evaluated on the 3/2-dealiased grid (Sec. "Scaled
transforms & dealiasing"): backward transforms (z then x) of u, w, dx b, bz,
dx u, uz, dx w, wz, pointwise products, forward transforms (x then z).

Pins: ``tests/test_oracle_rb.py`` (conductive steady state, linear onset at the
textbook Ra_c = 1707.76, k_c = 3.117, mean/BC invariants) and
``tests/test_oracle_advection.py`` (the advective terms of ``nonlinear``
against their closed form on a manufactured band-limited state, evaluated
pointwise by explicit sums).  Long nonlinear trajectories have no closed form:
they are pinned only through these pieces.
"""
import numpy as np

from . import bases
from .problem import TauProblem

RB_VARIABLES = ("b", "p", "u", "w", "bz", "uz", "wz")


def rb_problem(n_z, Ra, Pr=1.0):
    kappa = (Ra * Pr) ** -0.5
    nu = (Ra / Pr) ** -0.5
    pr = TauProblem(RB_VARIABLES, n_z, 0.0, 1.0)
    pr.add_equation("bz_def", L_terms=[("b", "dz", 1.0), ("bz", "I", -1.0)])
    pr.add_equation("uz_def", L_terms=[("u", "dz", 1.0), ("uz", "I", -1.0)])
    pr.add_equation("wz_def", L_terms=[("w", "dz", 1.0), ("wz", "I", -1.0)])
    pr.add_equation("b", M_terms=[("b", "I", 1.0)],
                    L_terms=[("b", "I", lambda k: kappa * k * k), ("bz", "dz", -kappa)])
    pr.add_equation("u", M_terms=[("u", "I", 1.0)],
                    L_terms=[("u", "I", lambda k: nu * k * k), ("uz", "dz", -nu),
                             ("p", "I", lambda k: 1j * k)])
    pr.add_equation("w", M_terms=[("w", "I", 1.0)],
                    L_terms=[("w", "I", lambda k: nu * k * k), ("wz", "dz", -nu),
                             ("p", "dz", 1.0), ("b", "I", -1.0)])
    pr.add_equation("div", L_terms=[("u", "I", lambda k: 1j * k), ("wz", "I", 1.0)])
    pr.add_bc("b", "left", value=lambda k: 1.0 if k == 0 else 0.0)
    pr.add_bc("b", "right", value=0.0)
    pr.add_bc("u", "left", value=0.0)
    pr.add_bc("u", "right", value=0.0)
    pr.add_bc("w", "left", value=0.0)
    pr.add_bc("w", "right", value=0.0, condition=lambda k: k != 0)
    pr.add_bc("p", "right", value=0.0, condition=lambda k: k == 0)
    return pr, kappa, nu


class RB2D:
    """2D Rayleigh-Benard on Fourier(x, N_x) x Chebyshev(z, N_z), dealias 3/2.

    State layout: complex array X[var, p, n] of T coefficients, var in
    RB_VARIABLES order, p = 0 .. N_x/2 - 1 the stored k_x >= 0 modes, n the
    Chebyshev mode.
    """

    def __init__(self, n_x, n_z, Ra, Pr=1.0, L_x=4.0, dealias=1.5, cheb_method="mmt", lu_method=None):
        self.Nx, self.Nz, self.Lx = int(n_x), int(n_z), float(L_x)
        self.Ra, self.Pr = float(Ra), float(Pr)
        self.problem, self.kappa, self.nu = rb_problem(self.Nz, self.Ra, self.Pr)
        self.S = len(RB_VARIABLES)
        self.P = self.Nx // 2
        self.kx = bases.fourier_wavenumbers(self.Nx, self.Lx)
        self.Ngx = int(round(dealias * self.Nx))
        self.Ngz = int(round(dealias * self.Nz))
        self.var = {v: i for i, v in enumerate(RB_VARIABLES)}
        self._mats = None
        # "mmt": explicit T_n(x_i) quadrature (default); "dct": scipy DCT, the
        # same definition summed in another order, with numpy's derivative
        # recurrence.  lu_method (timesteppers.PencilLU) picks the pencil
        # factorization: "auto" (dense LAPACK / SuperLU-COLAMD) or "natural"
        # (SuperLU in natural order).  The variants give rounding-floor
        # estimates: the same arithmetic summed in other orders.
        self.cheb_method = cheb_method
        self.lu_method = lu_method or ("natural" if cheb_method == "dct" else "auto")
        if cheb_method == "dct":
            self._cf, self._cb = bases.chebyshev_forward_dct, bases.chebyshev_backward_dct
        else:
            self._cf, self._cb = bases.chebyshev_forward, bases.chebyshev_backward

    # -- pencils ------------------------------------------------------------
    def matrices(self):
        if self._mats is None:
            self._mats = [self.problem.pencil_matrices(k) for k in self.kx]
        return self._mats

    def to_pencil(self, X, p):
        return X[:, p, :].reshape(-1)

    def from_pencils(self, vecs):
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        for p in range(self.P):
            X[:, p, :] = vecs[p].reshape(self.S, self.Nz)
        return X

    # -- transforms -----------------------------------------------------------
    def to_grid(self, c, n_gx=None, n_gz=None):
        """Coefficients c[p, n] -> real grid g[z, x] (z backward first, then x)."""
        n_gx = self.Ngx if n_gx is None else n_gx
        n_gz = self.Ngz if n_gz is None else n_gz
        gz = self._cb(c, n_gz, axis=1)                        # [p, zg]
        g = bases.fourier_backward(gz, n_gx, axis=0)          # [xg, zg]
        return g.T.copy()

    def to_coeff(self, g):
        """Real grid g[z, x] -> coefficients c[p, n] (x forward first, then z)."""
        fx = bases.fourier_forward(g, self.Nx, axis=1)        # [zg, p]
        c = self._cf(fx, self.Nz, axis=0)                     # [n, p]
        return c.T.copy()

    def dx(self, c):
        return 1j * self.kx[:, None] * c

    # -- nonlinear RHS ----------------------------------------------------------
    def nonlinear(self, X):
        """F per equation (T coefficients [p, n]) for the advective terms."""
        v = self.var
        g = lambda c: self.to_grid(c)
        u, w = g(X[v["u"]]), g(X[v["w"]])
        bx, bz = g(self.dx(X[v["b"]])), g(X[v["bz"]])
        ux, uz = g(self.dx(X[v["u"]])), g(X[v["uz"]])
        wx, wz = g(self.dx(X[v["w"]])), g(X[v["wz"]])
        return {
            "b": self.to_coeff(-(u * bx + w * bz)),
            "u": self.to_coeff(-(u * ux + w * uz)),
            "w": self.to_coeff(-(u * wx + w * wz)),
        }

    def rhs_vectors(self, X):
        """Pencil RHS vectors F~_p (left-preconditioned, boundary rows filled)."""
        F = self.nonlinear(X)
        return [self.problem.rhs_vector({e: F[e][p] for e in F}, self.kx[p])
                for p in range(self.P)]

    # -- initial state ------------------------------------------------------------
    def initial_state(self, noise, amplitude=1e-3):
        """b = 1 - z + A xi z (1 - z) on the scale-1 grid, bz = dz b, rest zero.

        ``noise`` is xi[z, x] on the N_z x N_x scale-1 grid (seeded standard
        normals drawn outside the oracle).
        """
        z = bases.chebyshev_grid(self.Nz)[:, None]
        b_grid = 1.0 - z + amplitude * noise * z * (1.0 - z)
        fx = bases.fourier_forward(b_grid, self.Nx, axis=1)          # [z, p]
        cb = self._cf(fx, self.Nz, axis=0).T                         # [p, n]
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        X[self.var["b"]] = cb
        if self.cheb_method == "dct":
            # second summation order: numpy's derivative recurrence (chebder)
            import numpy.polynomial.chebyshev as C
            d = C.chebder(cb, m=1, scl=2.0, axis=1)
            X[self.var["bz"], :, : self.Nz - 1] = d
        else:
            X[self.var["bz"]] = bases.chebyshev_derivative(cb, 0.0, 1.0, axis=1)
        return X

    def conductive_state(self):
        """b = 1 - z, bz = -1, p = z - z^2/2 - 1/2 (hydrostatic, p(1) = 0)."""
        z = bases.chebyshev_grid(self.Nz)
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        X[self.var["b"], 0] = bases.chebyshev_forward(1.0 - z, self.Nz)
        X[self.var["bz"], 0] = bases.chebyshev_forward(-np.ones_like(z), self.Nz)
        X[self.var["p"], 0] = bases.chebyshev_forward(z - 0.5 * z * z - 0.5, self.Nz)
        return X


def rb_onset_pencil(n_z, Ra, Pr, kx):
    """(M, L - F_X) for the linearisation about the conductive state.

    F_X is the Frechet derivative of the advective RHS at b = 1 - z, u = w = 0
    (the paper's F_X of Sec. "Nonlinear boundary value solver"): only
    -w dz(b_0) = +w survives, so the b equation gains the L term -w.  The
    eigenvalues s of  s M X + (L - F_X) X = 0  (Sec. "Eigenvalue solver")
    are the linear growth rates of convection.
    """
    pr, _, _ = rb_problem(n_z, Ra, Pr)
    for eq in pr.equations:
        if eq["name"] == "b":
            eq["L"].append(("w", "I", -1.0))
    return pr.pencil_matrices(kx)
