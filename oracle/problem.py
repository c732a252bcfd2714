"""Generic first-order tau pencil assembly in the plain Chebyshev-T basis (oracle).

Test infrastructure only.  Restates Sec. "Matrix construction" and Sec. "A
general sparse tau method" for one Fourier wavenumber k_x (one pencil):

* every equation is a sum of terms  coef(k_x) * op(variable)  split into the
  M group (multiplying the time derivative) and the L group, with
  op in {I, dz} along the Chebyshev axis (k_x factors such as i k_x or
  -k_x^2 are folded into coef), or a non-constant coefficient g(z) given by
  its Chebyshev coefficients (Sec. "Non-constant coefficients"): op = NCC(g)
  for g u, NCC(g, "dz") for dz(g u); the multiplication matrix in the T basis
  is (M_g)_{ij} = sum_n g_n (delta_{i,j+n} + delta_{i,|j-n|}) / 2 (Appendix,
  Chebyshev multiplication matrices), truncated to the N modes;
* an equation containing a z-derivative is "differential": each block is
  left-multiplied by the T-to-U conversion P^L (the dz blocks become the
  T-to-U derivative D^TU, times 2/(b-a) for the problem interval) and its last
  row is dropped (tau row, tau polynomial U_{N-1});
* an equation without a z-derivative keeps all N rows in the T basis;
* boundary-condition rows (interpolation vectors T_n(-1), T_n(1) times a
  variable) are appended after the equation rows, in L only (M rows zero),
  with their value on the right-hand side; a ``condition`` selects the
  pencils a row applies to (Sec. "Equation parsing": ``condition`` keyword).

Deliberate choices that keep this independent of any fast implementation:
blocks are concatenated variable by variable (no interleaving), the
unknowns are plain T coefficients (no Dirichlet recombination), and all
entries are complex (no real-ification).  Interleaving is a permutation and
recombination a change of variables, so a banded implementation must reach
the same solution to rounding.

Pins: ``tests/test_oracle_problem.py`` (polynomial exactness of the tau
solve, conductive steady state, dense-vs-sparse agreement).
"""
import numpy as np
import scipy.sparse as sps

from . import bases


class NCC:
    """Multiplication by g(z) = sum_n g[n] T_n, optionally followed by dz."""

    def __init__(self, g, after="I"):
        self.g = np.asarray(g, dtype=np.float64)
        self.after = after


def ncc_matrix(g, N):
    """(M_g)_{ij} = sum_n g_n (delta_{i,j+n} + delta_{i,|j-n|}) / 2, i, j < N."""
    M = np.zeros((N, N))
    for n, gn in enumerate(np.asarray(g, dtype=np.float64)):
        if gn == 0.0:
            continue
        for j in range(N):
            if j + n < N:
                M[j + n, j] += 0.5 * gn
            M[abs(j - n), j] += 0.5 * gn
    return M


class TauProblem:
    """A first-order system M dt(X) + L X = F on one Chebyshev axis per pencil."""

    def __init__(self, variables, n_z, a=0.0, b=1.0):
        self.variables = list(variables)
        self.S = len(self.variables)
        self.N = int(n_z)
        self.a, self.b = float(a), float(b)
        self.equations = []   # dicts: name, M terms, L terms, differential
        self.bcs = []         # dicts: var, side, value(kx), condition(kx)
        N = self.N
        self._I = sps.identity(N, format="csr", dtype=np.float64)
        self._PL = sps.csr_matrix(bases.cheb_P_L(N))
        self._DTU = sps.csr_matrix(bases.cheb_D_TU(N) * (2.0 / (self.b - self.a)))
        self._left = bases.cheb_left_vector(N)
        self._right = bases.cheb_right_vector(N)

    # -- declaration -------------------------------------------------------
    def add_equation(self, name, M_terms=(), L_terms=()):
        """Terms are (variable, op, coef) with op 'I' or 'dz' and coef a
        number or a function of k_x."""
        terms = list(M_terms) + list(L_terms)
        differential = any((op.after if isinstance(op, NCC) else op) == "dz" for (_, op, _) in terms)
        self.equations.append(dict(name=name, M=list(M_terms), L=list(L_terms),
                                   differential=differential))

    def add_bc(self, var, side, value=0.0, condition=None):
        self.bcs.append(dict(var=var, side=side, value=value, condition=condition))

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _eval(coef, kx):
        return complex(coef(kx)) if callable(coef) else complex(coef)

    def active_bcs(self, kx):
        return [bc for bc in self.bcs if bc["condition"] is None or bc["condition"](kx)]

    def equation_row_count(self, eq):
        return self.N - 1 if eq["differential"] else self.N

    def _block(self, eq, op, coef):
        if isinstance(op, NCC):
            Mg = sps.csr_matrix(ncc_matrix(op.g, self.N))
            if op.after == "dz":
                if not eq["differential"]:
                    raise ValueError("algebraic equation with a z-derivative")
                base = self._DTU @ Mg
            else:
                base = (self._PL @ Mg) if eq["differential"] else Mg
        elif eq["differential"]:
            base = self._PL if op == "I" else self._DTU
        else:
            if op != "I":
                raise ValueError("algebraic equation with a z-derivative")
            base = self._I
        blk = base * coef
        if eq["differential"]:
            blk = blk[: self.N - 1, :]
        return blk

    # -- assembly ----------------------------------------------------------
    def pencil_matrices(self, kx):
        """Return (M, L) as complex CSR matrices of size S*N for wavenumber kx."""
        S, N = self.S, self.N
        vidx = {v: i for i, v in enumerate(self.variables)}
        mats = {}
        for group in ("M", "L"):
            rows = []
            for eq in self.equations:
                nr = self.equation_row_count(eq)
                blocks = [sps.csr_matrix((nr, N), dtype=np.complex128) for _ in range(S)]
                for (var, op, coef) in eq[group]:
                    blocks[vidx[var]] = blocks[vidx[var]] + self._block(eq, op, self._eval(coef, kx))
                rows.append(blocks)
            for bc in self.active_bcs(kx):
                blocks = [sps.csr_matrix((1, N), dtype=np.complex128) for _ in range(S)]
                if group == "L":
                    vec = self._left if bc["side"] == "left" else self._right
                    blocks[vidx[bc["var"]]] = sps.csr_matrix(vec.reshape(1, N).astype(np.complex128))
                rows.append(blocks)
            mats[group] = sps.bmat(rows, format="csr")
        n_rows = mats["L"].shape[0]
        if n_rows != S * N:
            raise ValueError(f"pencil kx={kx}: {n_rows} rows for {S * N} unknowns")
        return mats["M"], mats["L"]

    def rhs_vector(self, F_eq, kx):
        """Assemble the pencil RHS from per-equation T coefficients.

        ``F_eq`` maps equation name -> length-N complex T coefficients (missing
        names are zero).  Differential equations get P^L and drop the last row;
        boundary rows carry their values.
        """
        N = self.N
        parts = []
        for eq in self.equations:
            f = F_eq.get(eq["name"])
            if f is None:
                parts.append(np.zeros(self.equation_row_count(eq), dtype=np.complex128))
                continue
            f = np.asarray(f, dtype=np.complex128)
            if eq["differential"]:
                parts.append((self._PL @ f)[: N - 1])
            else:
                parts.append(f.copy())
        for bc in self.active_bcs(kx):
            parts.append(np.array([self._eval(bc["value"], kx)], dtype=np.complex128))
        return np.concatenate(parts)

    def bc_vector(self, kx):
        """The RHS when every equation's F is zero (boundary values only)."""
        return self.rhs_vector({}, kx)


class LinearPencilSystem:
    """A TauProblem on a list of Fourier wavenumbers with F = boundary values
    plus an optional fixed forcing; the state is X[var, p, n] (T coefficients).

    Used to pin the timesteppers on linear problems with closed-form solutions.
    """

    def __init__(self, problem, kx, forcing=None):
        self.problem = problem
        self.kx = np.asarray(kx, dtype=np.float64)
        self.P = len(self.kx)
        self.S, self.N = problem.S, problem.N
        self.forcing = forcing  # optional callable X -> {eq: [p, n] coefficients}
        self._mats = None

    def matrices(self):
        if self._mats is None:
            self._mats = [self.problem.pencil_matrices(k) for k in self.kx]
        return self._mats

    def to_pencil(self, X, p):
        return X[:, p, :].reshape(-1)

    def from_pencils(self, vecs):
        X = np.zeros((self.S, self.P, self.N), dtype=np.complex128)
        for p in range(self.P):
            X[:, p, :] = vecs[p].reshape(self.S, self.N)
        return X

    def rhs_vectors(self, X):
        F = self.forcing(X) if self.forcing is not None else {}
        return [self.problem.rhs_vector({e: F[e][p] for e in F}, self.kx[p])
                for p in range(self.P)]
