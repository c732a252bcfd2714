"""Shared helpers for the GPU tests (no method arithmetic here)."""
import numpy as np


def rel_err(got, ref):
    """||got - ref||_2 / ||ref||_2, absolute when the reference norm < 1e-30."""
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(np.asarray(got) - np.asarray(ref))
    return d if nr < 1e-30 else d / nr


def field_errors(got, ref, names):
    return {v: rel_err(got[i], ref[i]) for i, v in enumerate(names)}


def oracle_floor(make_system, X0_fn, step_fn, nsteps):
    """Run the oracle twice (Chebyshev quadrature vs DCT summation) and return
    (reference, per-field rounding floor)."""
    out = []
    for method in ("mmt", "dct"):
        sysr = make_system(method)
        X = X0_fn(sysr)
        st = step_fn(sysr)
        for _ in range(nsteps):
            X = st.step(X, st.dt)
        out.append(X)
    return out[0], field_errors(out[1], out[0], NAMES)


def check_fields(got, ref, floor, bar):
    errs = field_errors(got, ref, NAMES)
    bad = {v: (errs[v], max(bar, 10 * floor[v])) for v in errs if errs[v] >= max(bar, 10 * floor[v])}
    assert not bad, {"errors": errs, "floor": floor, "failing (err, tol)": bad}


NAMES = ("b", "p", "u", "w", "bz", "uz", "wz")
