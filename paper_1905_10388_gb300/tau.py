"""Host-side assembly of preconditioned, interleaved tau pencils.

This is the problem assembler that sits above the C ABI: it turns a
first-order Fourier x Chebyshev problem into the per-pencil sparse matrices
M~_p = P^L M_p P^R and L~_p = P^L L_p P^R that ``sp_set_pencils`` takes,
plus the layout tables ``sp_set_layout`` takes.  It follows Sec. "Matrix
construction":

* equations with a z-derivative are left-preconditioned by the T-to-U
  conversion (derivatives become the banded T-to-U form) and lose their
  last row, which becomes a boundary (tau) row;
* variables with Dirichlet conditions are right-preconditioned by the
  Dirichlet recombination D_n = T_n - T_{n-2}, so boundary rows touch only
  modes 0 and 1 (Sec. "Banded boundary conditions", Appendix "Dirichlet
  recombination matrices");
* rows and columns are interleaved mode-major, variable-minor, which keeps
  the system banded with bandwidth O(S) (Sec. "Solving systems of
  equations").

Two GB300-specific choices go beyond the paper:

* real-ification: every variable and equation carries a phase i^q.  With
  x_true = i^{q_v} x~ and equation rows multiplied by i^{-q_e}, the RB
  pencils become real, so one real factor serves the real and imaginary
  parts of the complex right-hand side (half the FP64 work of a complex LU);
* row order: boundary rows come first (they touch modes 0 and 1), then the
  equation rows mode by mode in a per-problem order chosen to keep the
  lower bandwidth small, which is what partial pivoting fills.

Nothing here imports the oracle; the GPU tests compare the two.
"""
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np


def _as_fn(c):
    return c if callable(c) else (lambda k, c=c: c)


@dataclass
class Term:
    var: str
    op: str            # "I", "dz", "ncc" (g u) or "nccdz" (dz(g u))
    coef: object       # number or function of the wavenumber(s) (evaluated on arrays)
    ncc: Optional[Sequence[float]] = None   # Chebyshev coefficients of g(z) for the ncc ops


@dataclass
class Equation:
    name: str
    M: List[Term] = field(default_factory=list)
    L: List[Term] = field(default_factory=list)
    phase: int = 0     # rows are multiplied by i^(-phase)

    @property
    def differential(self):
        return any(t.op in ("dz", "nccdz") for t in self.M + self.L)


@dataclass
class BCAlternative:
    var: str
    side: str          # "left" (z = a) or "right" (z = b)
    value: object = 0.0
    condition: Optional[Callable] = None    # wavenumber arrays -> boolean array
    phase: int = 0


@dataclass
class BCSlot:
    """One boundary row; exactly one alternative applies to each pencil."""
    alternatives: List[BCAlternative]


# --- 1D operator entries on N Chebyshev modes (native interval [-1, 1]) ------

def _conv_entries(N):
    """T-to-U conversion P^L: (row i, col j, value)."""
    out = []
    for j in range(N):
        out.append((j, j, 1.0 if j == 0 else 0.5))
        if j >= 2:
            out.append((j - 2, j, -0.5))
    return out


def _dtu_entries(N, scale):
    return [(j - 1, j, scale * j) for j in range(1, N)]


def _ident_entries(N):
    return [(j, j, 1.0) for j in range(N)]


def _ncc_entries(g, N):
    """Multiplication by g(z) = sum_n g_n T_n in the T basis (Sec. "Non-
    constant coefficients"; T_n T_j = (T_{j+n} + T_{|j-n|}) / 2), truncated to
    N modes: bandwidth len(g) - 1 above and below the diagonal."""
    acc = {}
    for n, gn in enumerate(np.asarray(g, dtype=np.float64)):
        if gn == 0.0:
            continue
        for j in range(N):
            for i in (j + n, abs(j - n)):
                if i < N:
                    acc[(i, j)] = acc.get((i, j), 0.0) + 0.5 * gn
    return [(i, j, v) for (i, j), v in acc.items() if v != 0.0]


def _compose(a, b):
    """Entries of the product A B of two sparse operators given as entries."""
    rows = {}
    for (i, k, v) in a:
        rows.setdefault(k, []).append((i, v))
    acc = {}
    for (k, j, w) in b:
        for (i, v) in rows.get(k, []):
            acc[(i, j)] = acc.get((i, j), 0.0) + v * w
    return [(i, j, v) for (i, j), v in acc.items() if v != 0.0]


def _recombine(entries, N):
    """Right-multiply an operator (list of entries) by the Dirichlet
    recombination P^R, (P^R)_{mj} = delta_mj - delta_{m,j-2} [j > 1]:
    column j of A P^R is A[:, j] - A[:, j-2] for j >= 2."""
    cols = {}
    for (i, m, v) in entries:
        cols.setdefault(m, []).append((i, v))
    out = []
    for j in range(N):
        for (i, v) in cols.get(j, []):
            out.append((i, j, v))
        if j >= 2:
            for (i, v) in cols.get(j - 2, []):
                out.append((i, j, -v))
    return out


def _bc_vector(N, side, recombined):
    if recombined:
        vals = np.zeros(N)
        vals[0] = 1.0
        if N > 1:
            vals[1] = -1.0 if side == "left" else 1.0
    else:
        vals = (-1.0) ** np.arange(N) if side == "left" else np.ones(N)
    return [(0, j, float(vals[j])) for j in range(N) if vals[j] != 0.0]


class PencilProblem:
    """First-order problem on Fourier(x) x Chebyshev(z in [a, b]) pencils."""

    def __init__(self, variables: Sequence[str], equations: Sequence[Equation],
                 bc_slots: Sequence[BCSlot], recombine: Sequence[str] = (),
                 var_phase: Optional[dict] = None, row_order: Optional[Sequence[str]] = None,
                 a=0.0, b=1.0):
        self.variables = list(variables)
        self.S = len(self.variables)
        self.equations = list(equations)
        if len(self.equations) != self.S:
            raise ValueError("need as many equations as variables")
        self.bc_slots = list(bc_slots)
        self.recombine = set(recombine)
        self.var_phase = dict(var_phase or {})
        self.eq_order = list(row_order) if row_order else [e.name for e in self.equations]
        self.a, self.b = float(a), float(b)
        self.vslot = {v: i for i, v in enumerate(self.variables)}
        self.eq_by_name = {e.name: e for e in self.equations}
        n_diff = sum(e.differential for e in self.equations)
        if n_diff != len(self.bc_slots):
            raise ValueError("one boundary row per differential equation is required")

    # -- layout ----------------------------------------------------------------
    def layout(self, N):
        """col_map[v, m], row_map[e, m] (-1 = dropped tau row), bc row indices."""
        S = self.S
        col_map = np.zeros((S, N), dtype=np.int32)
        for v in range(S):
            col_map[v] = np.arange(N) * S + v
        row_map = -np.ones((S, N), dtype=np.int32)
        nbc = len(self.bc_slots)
        bc_rows = np.arange(nbc, dtype=np.int32)
        r = nbc
        eidx = {e.name: i for i, e in enumerate(self.equations)}
        for m in range(N):
            for name in self.eq_order:
                e = self.eq_by_name[name]
                if e.differential and m == N - 1:
                    continue
                row_map[eidx[name], m] = r
                r += 1
        assert r == S * N
        return col_map, row_map, bc_rows

    # -- assembly ----------------------------------------------------------------
    def _term_entries(self, eq, term, N):
        zscale = 2.0 / (self.b - self.a)
        if term.op in ("ncc", "nccdz"):
            g = _ncc_entries(term.ncc, N)
            if eq.differential:
                left = _conv_entries(N) if term.op == "ncc" else _dtu_entries(N, zscale)
                base = _compose(left, g)
                base = [(i, j, v) for (i, j, v) in base if i < N - 1]
            else:
                if term.op != "ncc":
                    raise ValueError("algebraic equation with a z-derivative")
                base = g
        elif eq.differential:
            base = _conv_entries(N) if term.op == "I" else _dtu_entries(N, zscale)
            base = [(i, j, v) for (i, j, v) in base if i < N - 1]
        else:
            if term.op != "I":
                raise ValueError("algebraic equation with a z-derivative")
            base = _ident_entries(N)
        if term.var in self.recombine:
            base = _recombine(base, N)
        return base

    def pattern(self, N):
        """Structural entries: list of (row, col, group, term-key, base value)."""
        col_map, row_map, bc_rows = self.layout(N)
        ents = []
        for ei, eq in enumerate(self.equations):
            for group in ("M", "L"):
                for ti, term in enumerate(getattr(eq, group)):
                    v = self.vslot[term.var]
                    for (i, j, val) in self._term_entries(eq, term, N):
                        ents.append((row_map[ei, i], col_map[v, j], group, ("eq", ei, group, ti), val))
        for si, slot in enumerate(self.bc_slots):
            for ai, alt in enumerate(slot.alternatives):
                v = self.vslot[alt.var]
                for (_, j, val) in _bc_vector(N, alt.side, alt.var in self.recombine):
                    ents.append((bc_rows[si], col_map[v, j], "L", ("bc", si, ai), val))
        return ents

    def _phase(self, q):
        return 1j ** (q % 4)

    def build(self, N, wavenumbers, values=True):
        """Assemble every pencil on a shared (union) CSR pattern.

        ``wavenumbers`` gives one entry per pencil: an array of k_x (one
        Fourier axis) or a tuple of arrays (k_x, k_y) (two Fourier axes);
        coefficient functions, boundary values and conditions are evaluated
        on those arrays.  Returns a dict with indptr, indices, the layout
        tables, the band widths, bc_values [P, nbc] complex and a function
        ``values(p0, p1)`` -> (M, L) real [p1 - p0, nnz] for a range of
        pencils (and, when ``values`` is true, M and L for all pencils).
        """
        k = tuple(np.asarray(a, dtype=np.float64) for a in wavenumbers) if isinstance(wavenumbers, tuple) \
            else np.asarray(wavenumbers, dtype=np.float64)
        P = len(k[0]) if isinstance(k, tuple) else len(k)
        S, n = self.S, self.S * N
        ents = self.pattern(N)
        rows = np.array([e[0] for e in ents], dtype=np.int64)
        cols = np.array([e[1] for e in ents], dtype=np.int64)
        key = rows * n + cols
        ukey, inv = np.unique(key, return_inverse=True)
        urow, ucol = ukey // n, ukey % n
        nnz = len(ukey)
        indptr = np.zeros(n + 1, dtype=np.int32)
        np.add.at(indptr, urow + 1, 1)
        indptr = np.cumsum(indptr).astype(np.int32)
        indices = ucol.astype(np.int32)
        nbc = len(self.bc_slots)
        vq = {v: self.var_phase.get(v, 0) for v in self.variables}

        def per_pencil(c, dtype=np.complex128):
            return np.broadcast_to(np.asarray(_as_fn(c)(k), dtype=dtype), (P,))

        # the boundary alternative that applies to each pencil
        active = np.zeros((nbc, P), dtype=np.int64)
        for si, slot in enumerate(self.bc_slots):
            hits = np.stack([np.ones(P, bool) if a.condition is None else per_pencil(a.condition, bool)
                             for a in slot.alternatives])
            if not np.all(hits.sum(axis=0) == 1):
                raise ValueError(f"boundary slot {si} needs exactly one alternative on every pencil")
            active[si] = np.argmax(hits, axis=0)
        # every entry belongs to one term (or one boundary alternative); its
        # value on pencil p is scale[term, p] * base value
        keys, key_index = [], {}
        ent_key = np.empty(len(ents), dtype=np.int64)
        for t, e in enumerate(ents):
            kk = e[3]
            if kk not in key_index:
                key_index[kk] = len(keys)
                keys.append(kk)
            ent_key[t] = key_index[kk]
        base = np.array([e[4] for e in ents], dtype=np.float64)
        is_M = np.array([e[2] == "M" for e in ents])
        scale = np.zeros((len(keys), P), dtype=np.complex128)
        for ki, kk in enumerate(keys):
            if kk[0] == "eq":
                _, ei, g, ti = kk
                eq = self.equations[ei]
                term = getattr(eq, g)[ti]
                scale[ki] = per_pencil(term.coef) * self._phase(vq[term.var] - eq.phase)
            else:
                _, si, ai = kk
                alt = self.bc_slots[si].alternatives[ai]
                scale[ki] = np.where(active[si] == ai, self._phase(vq[alt.var] - alt.phase), 0.0)
        bcv = np.zeros((P, nbc), dtype=np.complex128)
        for si, slot in enumerate(self.bc_slots):
            for ai, alt in enumerate(slot.alternatives):
                bcv[:, si] += np.where(active[si] == ai, per_pencil(alt.value) * self._phase(-alt.phase), 0.0)
        # value maps: nnz x keys (base values summed per structural slot)
        import scipy.sparse as sps
        maps = []
        for mask in (is_M, ~is_M):
            idx = np.nonzero(mask)[0]
            maps.append(sps.csr_matrix((base[idx], (inv[idx], ent_key[idx])), shape=(nnz, len(keys))))

        scale_re = np.ascontiguousarray(scale.real)
        scale_im = np.ascontiguousarray(scale.imag)

        def pencil_values(p0, p1):
            out = []
            for A in maps:
                Xr = (A @ scale_re[:, p0:p1]).T                     # [p1 - p0, nnz]
                Xi = A @ scale_im[:, p0:p1]
                if np.abs(Xi).max(initial=0) > 1e-14 * max(1.0, np.abs(Xr).max(initial=0)):
                    raise ValueError("pencil is not real under the given phases")
                out.append(np.ascontiguousarray(Xr))
            return tuple(out)

        col_map, row_map, bc_rows = self.layout(N)
        d = ucol - urow
        res = dict(
            n=n, N=N, S=S, P=P, indptr=indptr, indices=indices, values=pencil_values,
            bc_values=bcv, bc_rows=bc_rows, col_map=col_map, row_map=row_map,
            kl=int(max(0, -d.min())), ku=int(max(0, d.max())),
            var_recombine=np.array([v in self.recombine for v in self.variables], np.int32),
            var_phase=np.array([vq[v] for v in self.variables], np.int32),
            eq_differential=np.array([e.differential for e in self.equations], np.int32),
            eq_phase=np.array([e.phase for e in self.equations], np.int32),
        )
        if values:
            res["M"], res["L"] = pencil_values(0, P)
        return res
