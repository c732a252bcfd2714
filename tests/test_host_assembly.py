"""Host-side checks without a GPU.

* The product's pencil assembler (interleaved, Dirichlet-recombined,
  real-ified, boundary rows on top) must give the same solution as the
  oracle's plain complex T-basis pencils: interleaving is a permutation and
  recombination / phases a change of variables (Sec. "Matrix construction").
  The right-hand side is placed exactly as the solve kernel's prologue does
  (row_map, T-to-U conversion, phases, boundary values) and the solution is
  mapped back as its epilogue does (col_map, x_m = x~_m - x~_{m+2}, phases).
* libspectau.so exports every entry point declared in include/spectau.h.
"""
import os
import re

import numpy as np
import pytest

from oracle import rb as orb
from paper_1905_10388_gb300 import rb as prb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _csr_dense(indptr, indices, vals, n):
    A = np.zeros((n, n))
    for r in range(n):
        for e in range(indptr[r], indptr[r + 1]):
            A[r, indices[e]] += vals[e]
    return A


def _place_rhs(asm, p, F_eq, eq_names):
    """RHS vector as assembled by the solve kernel's prologue."""
    N, S, n = asm["N"], asm["S"], asm["n"]
    B = np.zeros(n, complex)
    for e, name in enumerate(eq_names):
        f = F_eq.get(name)
        if f is None:
            continue
        for m in range(N):
            row = asm["row_map"][e, m]
            if row < 0:
                continue
            if asm["eq_differential"][e]:
                u = f[m] * (1.0 if m == 0 else 0.5) - (0.5 * f[m + 2] if m + 2 < N else 0.0)
            else:
                u = f[m]
            B[row] += (1j ** (-asm["eq_phase"][e])) * u
    for q, row in enumerate(asm["bc_rows"]):
        B[row] += asm["bc_values"][p, q]
    return B


def _unmap(asm, x, var_names):
    N = asm["N"]
    out = {}
    for v, name in enumerate(var_names):
        c = np.array([x[asm["col_map"][v, m]] for m in range(N)])
        if asm["var_recombine"][v]:
            c[: N - 2] -= c[2:]
        out[name] = (1j ** asm["var_phase"][v]) * c
    return out


@pytest.mark.parametrize("N", [8, 12, 17])
@pytest.mark.parametrize("kx", [0.0, 1.5707963267948966, 4.71238898038469])
def test_assembler_matches_oracle_pencil(N, kx):
    Ra, Pr, a = 1e5, 1.0, 3e-3
    prob = prb.rb_pencil_problem(Ra, Pr)
    asm = prob.build(N, np.array([kx]))
    n = asm["n"]
    At = _csr_dense(asm["indptr"], asm["indices"], asm["M"][0] + a * asm["L"][0], n)
    opr, _, _ = orb.rb_problem(N, Ra, Pr)
    M, L = opr.pencil_matrices(kx)
    rng = np.random.default_rng(int(N * 100 + kx * 10))
    F = {e: rng.standard_normal(N) + 1j * rng.standard_normal(N) for e in ("b", "u", "w")}
    X_ref = np.linalg.solve((M + a * L).toarray(), opr.rhs_vector(F, kx))
    names_eq = [e.name for e in prob.equations]
    B = _place_rhs(asm, 0, F, names_eq)
    x = np.linalg.solve(At, B.real) + 1j * np.linalg.solve(At, B.imag)
    got = _unmap(asm, x, prob.variables)
    for i, v in enumerate(orb.RB_VARIABLES):
        ref = X_ref[i * N:(i + 1) * N]
        assert np.abs(got[v] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), v


@pytest.mark.parametrize("k", [(0.0, 0.0), (1.5707963267948966, 0.0), (0.0, -3.14159265358979),
                               (4.71238898038469, 1.5707963267948966)])
def test_3d_assembler_matches_oracle_pencil(k):
    from oracle import rb3d as orb3
    N, Ra, Pr, a = 12, 1e5, 1.0, 3e-3
    prob = prb.rb3d_pencil_problem(Ra, Pr)
    asm = prob.build(N, (np.array([k[0]]), np.array([k[1]])))
    n = asm["n"]
    At = _csr_dense(asm["indptr"], asm["indices"], asm["M"][0] + a * asm["L"][0], n)
    opr, _, _ = orb3.rb3d_problem(N, Ra, Pr)
    M, L = opr.pencil_matrices(k)
    rng = np.random.default_rng(5)
    F = {e: rng.standard_normal(N) + 1j * rng.standard_normal(N) for e in ("b", "u", "v", "w")}
    X_ref = np.linalg.solve((M + a * L).toarray(), opr.rhs_vector(F, k))
    B = _place_rhs(asm, 0, F, [e.name for e in prob.equations])
    x = np.linalg.solve(At, B.real) + 1j * np.linalg.solve(At, B.imag)
    got = _unmap(asm, x, prob.variables)
    for i, v in enumerate(orb3.RB3D_VARIABLES):
        ref = X_ref[i * N:(i + 1) * N]
        assert np.abs(got[v] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), v
    assert (asm["kl"], asm["ku"]) == (9, 29)


def test_band_widths_of_rb_ordering():
    asm = prb.rb_pencil_problem(1e6).build(32, np.array([0.0, 1.0]))
    assert (asm["kl"], asm["ku"]) == (7, 22)
    assert np.all(np.isfinite(asm["M"])) and np.all(np.isfinite(asm["L"]))


def test_matrices_are_real_under_phases():
    prob = prb.rb_pencil_problem(1e6)
    prob.var_phase = {}            # without the phases the pencils are complex
    with pytest.raises(ValueError):
        prob.build(8, np.array([1.0]))


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "spectau.h")).read()
    return sorted(set(re.findall(r"^\s*(?:sp_status|const char\*)\s+(sp_\w+)\(", hdr, re.M)))


def test_library_exports_every_declared_symbol():
    import paper_1905_10388_gb300 as pk
    lib_path = pk.build()
    import ctypes
    L = ctypes.CDLL(lib_path)
    syms = _declared_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(L, s), s
    from paper_1905_10388_gb300 import _lib
    assert sorted(_lib.EXPORTS) == syms
