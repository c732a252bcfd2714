"""Fisher-KPP reaction-diffusion in first-order tau form (oracle; test
infrastructure).

The overview example of Sec. "Codebase structure": u(x, z, t) on a channel
periodic in x (Fourier) and bounded in z (Chebyshev, [0, 1]), with

    dt(u) - D (dx dx u + dz uz) = R u (1 - u),     uz = dz(u),
    uz(0) = uz(1) = 0 (Neumann walls).

In the IVP form M dt(X) + L X = F(X) (Sec. "Initial value solver") with
X = (u, uz) the reaction's linear part goes to L and its quadratic part is
the explicit right-hand side:

    uz_def:  dz(u) - uz = 0
    u:       dt(u) - D (dx dx u + dz uz) - R u = -R u u

The product is evaluated on the 3/2-dealiased grid (Sec. "Scaled transforms
& dealiasing"): backward transforms (z then x) of u, pointwise square,
forward transforms (x then z).

Pins: ``tests/test_oracle_fisher.py`` (a uniform state follows the logistic
equation's closed form at the scheme's order; with R = 0 a diffusion mode
decays at D (k^2 + pi^2) to spectral accuracy; the dealiased square equals
the exact truncated product of the two expansions).
"""
import numpy as np

from . import bases
from .problem import TauProblem

FISHER_VARIABLES = ("u", "uz")


def fisher_problem(n_z, D, R):
    pr = TauProblem(FISHER_VARIABLES, n_z, 0.0, 1.0)
    pr.add_equation("uz_def", L_terms=[("u", "dz", 1.0), ("uz", "I", -1.0)])
    pr.add_equation("u", M_terms=[("u", "I", 1.0)],
                    L_terms=[("u", "I", lambda k: D * k * k - R), ("uz", "dz", -D)])
    pr.add_bc("uz", "left", value=0.0)
    pr.add_bc("uz", "right", value=0.0)
    return pr


class FisherKPP:
    """Fisher-KPP on Fourier(x, N_x) x Chebyshev(z, N_z), dealias 3/2.

    State: complex X[var, p, n], var in FISHER_VARIABLES order, p the stored
    k_x >= 0 modes, n the Chebyshev mode.
    """

    def __init__(self, n_x, n_z, D=0.1, R=1.0, L_x=2 * np.pi, dealias=1.5, lu_method="auto"):
        self.Nx, self.Nz, self.Lx = int(n_x), int(n_z), float(L_x)
        self.D, self.R = float(D), float(R)
        self.problem = fisher_problem(self.Nz, self.D, self.R)
        self.S = len(FISHER_VARIABLES)
        self.P = self.Nx // 2
        self.kx = bases.fourier_wavenumbers(self.Nx, self.Lx)
        self.Ngx = int(round(dealias * self.Nx))
        self.Ngz = int(round(dealias * self.Nz))
        self.var = {v: i for i, v in enumerate(FISHER_VARIABLES)}
        self.lu_method = lu_method
        self._mats = None

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

    def to_grid(self, c, n_gx=None, n_gz=None):
        """Coefficients c[p, n] -> real grid g[z, x] (z first, then x)."""
        n_gx = self.Ngx if n_gx is None else n_gx
        n_gz = self.Ngz if n_gz is None else n_gz
        gz = bases.chebyshev_backward(c, n_gz, axis=1)
        return bases.fourier_backward(gz, n_gx, axis=0).T.copy()

    def to_coeff(self, g):
        """Real grid g[z, x] -> coefficients c[p, n] (x first, then z)."""
        fx = bases.fourier_forward(g, self.Nx, axis=1)
        return bases.chebyshev_forward(fx, self.Nz, axis=0).T.copy()

    def nonlinear(self, X):
        u = self.to_grid(X[self.var["u"]])
        return {"u": self.to_coeff(-self.R * u * u)}

    def rhs_vectors(self, X):
        F = self.nonlinear(X)
        return [self.problem.rhs_vector({"u": F["u"][p]}, self.kx[p]) for p in range(self.P)]

    def initial_state(self, u_grid):
        """u from its values on the scale-1 grid [z, x], uz = dz u."""
        X = np.zeros((self.S, self.P, self.Nz), dtype=np.complex128)
        cu = self.to_coeff(np.asarray(u_grid, dtype=np.float64))
        X[self.var["u"]] = cu
        X[self.var["uz"]] = bases.chebyshev_derivative(cu, 0.0, 1.0, axis=1)
        return X
