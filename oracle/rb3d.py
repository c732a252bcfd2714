"""Three-dimensional Rayleigh-Benard convection in first-order tau form (oracle;
test infrastructure).

Fourier x (real data: stored k_x >= 0 modes), Fourier y (complex axis, FFT
order, Nyquist slot zero), Chebyshev z in [0, 1].  The 2D system of
``oracle.rb`` with the y-velocity v, its derivative vz, the v equation and
the y-derivatives; X = (b, p, u, v, w, bz, uz, vz, wz):

    bz_def:  dz(b) - bz = 0        uz_def: dz(u) - uz = 0
    vz_def:  dz(v) - vz = 0        wz_def: dz(w) - wz = 0
    b:  dt(b) - kappa (lap_h b + dz bz)         = -(u dx b + v dy b + w bz)
    u:  dt(u) - nu (lap_h u + dz uz) + dx p     = -(u dx u + v dy u + w uz)
    v:  dt(v) - nu (lap_h v + dz vz) + dy p     = -(u dx v + v dy v + w vz)
    w:  dt(w) - nu (lap_h w + dz wz) + dz p - b = -(u dx w + v dy w + w wz)
    div: dx u + dy v + wz = 0

    b(0) = 1, b(1) = 0, u = v = 0 at both walls, w(0) = 0, and w(1) = 0 for
    (k_x, k_y) != 0 or the gauge p(1) = 0 at k_x = k_y = 0.

One pencil per (k_y slot, k_x) pair, pencil index p = i_y (N_x / 2) + i_x.
Transforms follow Sec. "Scaled transforms & dealiasing" with the order z, y,
x backward and x, y, z forward, on the 3/2 grid.

Pins: ``tests/test_oracle_rb3d.py`` (y-transform modes and round trip, the
reduction to the 2D system for y-independent states, rotation invariance of
the linear growth rates, the conductive steady state) and
``tests/test_oracle_advection.py`` (the advective terms against their closed
form on a manufactured band-limited state).
"""
import numpy as np

from . import bases
from .problem import TauProblem

RB3D_VARIABLES = ("b", "p", "u", "v", "w", "bz", "uz", "vz", "wz")


def rb3d_problem(n_z, Ra, Pr=1.0):
    """The 3D pencil problem; coefficient functions take k = (k_x, k_y)."""
    kappa = (Ra * Pr) ** -0.5
    nu = (Ra / Pr) ** -0.5
    k2 = lambda k: k[0] * k[0] + k[1] * k[1]
    pr = TauProblem(RB3D_VARIABLES, n_z, 0.0, 1.0)
    for f in ("b", "u", "v", "w"):
        pr.add_equation(f + "z_def", L_terms=[(f, "dz", 1.0), (f + "z", "I", -1.0)])
    pr.add_equation("b", M_terms=[("b", "I", 1.0)],
                    L_terms=[("b", "I", lambda k: kappa * k2(k)), ("bz", "dz", -kappa)])
    pr.add_equation("u", M_terms=[("u", "I", 1.0)],
                    L_terms=[("u", "I", lambda k: nu * k2(k)), ("uz", "dz", -nu),
                             ("p", "I", lambda k: 1j * k[0])])
    pr.add_equation("v", M_terms=[("v", "I", 1.0)],
                    L_terms=[("v", "I", lambda k: nu * k2(k)), ("vz", "dz", -nu),
                             ("p", "I", lambda k: 1j * k[1])])
    pr.add_equation("w", M_terms=[("w", "I", 1.0)],
                    L_terms=[("w", "I", lambda k: nu * k2(k)), ("wz", "dz", -nu),
                             ("p", "dz", 1.0), ("b", "I", -1.0)])
    pr.add_equation("div", L_terms=[("u", "I", lambda k: 1j * k[0]), ("v", "I", lambda k: 1j * k[1]),
                                    ("wz", "I", 1.0)])
    mean = lambda k: k[0] == 0 and k[1] == 0
    pr.add_bc("b", "left", value=lambda k: 1.0 if mean(k) else 0.0)
    pr.add_bc("b", "right", value=0.0)
    for f in ("u", "v"):
        pr.add_bc(f, "left", value=0.0)
        pr.add_bc(f, "right", value=0.0)
    pr.add_bc("w", "left", value=0.0)
    pr.add_bc("w", "right", value=0.0, condition=lambda k: not mean(k))
    pr.add_bc("p", "right", value=0.0, condition=mean)
    return pr, kappa, nu


class RB3D:
    """3D Rayleigh-Benard on Fourier(x) x Fourier(y) x Chebyshev(z), dealias 3/2.

    State: complex X[var, p, n], var in RB3D_VARIABLES order, p = i_y K + i_x
    (K = N_x / 2 stored k_x >= 0 modes, i_y the FFT-order k_y slot), n the
    Chebyshev mode.
    """

    def __init__(self, n_x, n_y, n_z, Ra, Pr=1.0, L_x=4.0, L_y=4.0, dealias=1.5, lu_method="auto",
                 cheb_method="mmt"):
        self.Nx, self.Ny, self.Nz = int(n_x), int(n_y), int(n_z)
        self.Lx, self.Ly = float(L_x), float(L_y)
        self.Ra, self.Pr = float(Ra), float(Pr)
        self.problem, self.kappa, self.nu = rb3d_problem(self.Nz, self.Ra, self.Pr)
        self.S = len(RB3D_VARIABLES)
        self.K = self.Nx // 2
        self.P = self.Ny * self.K
        kx = bases.fourier_wavenumbers(self.Nx, self.Lx)
        ky = bases.fourier_c_wavenumbers(self.Ny, self.Ly)
        self.kx = np.tile(kx, self.Ny)                  # per pencil
        self.ky = np.repeat(ky, self.K)
        self.Ngx = int(round(dealias * self.Nx))
        self.Ngy = int(round(dealias * self.Ny))
        self.Ngz = int(round(dealias * self.Nz))
        self.var = {v: i for i, v in enumerate(RB3D_VARIABLES)}
        self.lu_method = lu_method
        # "mmt": explicit T_n(x_i) quadrature (default); "dct": scipy DCT, the
        # same definition summed in another order, with numpy's derivative
        # recurrence for the initial bz (as in the 2D oracle): a rounding-floor
        # variant
        self.cheb_method = cheb_method
        if cheb_method == "dct":
            self._cf, self._cb = bases.chebyshev_forward_dct, bases.chebyshev_backward_dct
        else:
            self._cf, self._cb = bases.chebyshev_forward, bases.chebyshev_backward
        self._mats = None

    # -- pencils ------------------------------------------------------------
    def wavenumber(self, p):
        return (float(self.kx[p]), float(self.ky[p]))

    def matrices(self):
        if self._mats is None:
            self._mats = [self.problem.pencil_matrices(self.wavenumber(p)) for p in range(self.P)]
        return self._mats

    def to_pencil(self, X, p):
        return X[:, p, :].reshape(-1)

    def from_pencils(self, vecs):
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        for p in range(self.P):
            X[:, p, :] = vecs[p].reshape(self.S, self.Nz)
        return X

    # -- transforms -----------------------------------------------------------
    def to_grid(self, c, n_gx=None, n_gy=None, n_gz=None):
        """Coefficients c[p, n] -> real grid g[z, y, x] (z, then y, then x)."""
        n_gx = self.Ngx if n_gx is None else n_gx
        n_gy = self.Ngy if n_gy is None else n_gy
        n_gz = self.Ngz if n_gz is None else n_gz
        c3 = np.asarray(c).reshape(self.Ny, self.K, self.Nz)
        gz = self._cb(c3, n_gz, axis=2)                           # [iy, ix, zg]
        gy = bases.fourier_c_backward(gz, n_gy, axis=0)           # [yg, ix, zg]
        g = bases.fourier_backward(gy, n_gx, axis=1)              # [yg, xg, zg]
        return np.transpose(g, (2, 0, 1)).copy()

    def to_coeff(self, g):
        """Real grid g[z, y, x] -> coefficients c[p, n] (x, then y, then z)."""
        fx = bases.fourier_forward(g, self.Nx, axis=2)            # [z, y, ix]
        fy = bases.fourier_c_forward(fx, self.Ny, axis=1)         # [z, iy, ix]
        c = self._cf(fy, self.Nz, axis=0)                         # [n, iy, ix]
        return np.transpose(c, (1, 2, 0)).reshape(self.P, self.Nz).copy()

    def dx(self, c):
        return 1j * self.kx[:, None] * c

    def dy(self, c):
        return 1j * self.ky[:, None] * c

    # -- nonlinear RHS ----------------------------------------------------------
    def nonlinear(self, X):
        """F per equation (T coefficients [p, n]) of the advective terms."""
        v = self.var
        g = self.to_grid
        U = {f: g(X[v[f]]) for f in ("u", "v", "w")}
        out = {}
        for e in ("b", "u", "v", "w"):
            c = X[v[e]]
            adv = U["u"] * g(self.dx(c)) + U["v"] * g(self.dy(c)) + U["w"] * g(X[v[e + "z"]])
            out[e] = self.to_coeff(-adv)
        return out

    def rhs_vectors(self, X):
        F = self.nonlinear(X)
        return [self.problem.rhs_vector({e: F[e][p] for e in F}, self.wavenumber(p)) for p in range(self.P)]

    # -- states ---------------------------------------------------------------------
    def initial_state(self, noise, amplitude=1e-3):
        """b = 1 - z + A xi z (1 - z) on the scale-1 grid (xi[z, y, x]), bz = dz b."""
        z = bases.chebyshev_grid(self.Nz)[:, None, None]
        b_grid = 1.0 - z + amplitude * np.asarray(noise) * z * (1.0 - z)
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        cb = self.to_coeff(b_grid)
        X[self.var["b"]] = cb
        if self.cheb_method == "dct":
            import numpy.polynomial.chebyshev as C
            X[self.var["bz"], :, : self.Nz - 1] = C.chebder(cb, m=1, scl=2.0, axis=1)
        else:
            X[self.var["bz"]] = bases.chebyshev_derivative(cb, 0.0, 1.0, axis=1)
        return X

    def conductive_state(self):
        """b = 1 - z, bz = -1, p = z - z^2/2 - 1/2 in the k = 0 pencil."""
        z = bases.chebyshev_grid(self.Nz)
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        X[self.var["b"], 0] = bases.chebyshev_forward(1.0 - z, self.Nz)
        X[self.var["bz"], 0] = bases.chebyshev_forward(-np.ones_like(z), self.Nz)
        X[self.var["p"], 0] = bases.chebyshev_forward(z - 0.5 * z * z - 0.5, self.Nz)
        return X


def rb3d_onset_pencil(n_z, Ra, Pr, k):
    """(M, L - F_X) of the linearisation about the conductive state at the
    wavenumber k = (k_x, k_y) (see ``oracle.rb.rb_onset_pencil``)."""
    pr, _, _ = rb3d_problem(n_z, Ra, Pr)
    for eq in pr.equations:
        if eq["name"] == "b":
            eq["L"].append(("w", "I", -1.0))
    return pr.pencil_matrices(k)
