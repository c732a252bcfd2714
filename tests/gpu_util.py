"""Shared helpers for the GPU tests (no method arithmetic here)."""
import json
import os

import numpy as np


def rel_err(got, ref):
    """||got - ref||_2 / ||ref||_2, absolute when the reference norm < 1e-30."""
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(np.asarray(got) - np.asarray(ref))
    return d if nr < 1e-30 else d / nr


def field_errors(got, ref, names):
    return {v: rel_err(got[i], ref[i]) for i, v in enumerate(names)}


# Oracle variants whose spread estimates the rounding floor of each field:
# (Chebyshev summation, pencil factorization) other than the reference's
# ("mmt", "auto").  The solve dominates the spread of fields such as bz,
# whose relative error is set by the conditioning of the pencil matrices.
FLOOR_VARIANTS = (("dct", "natural"), ("mmt", "natural"), ("dct", "auto"))


def oracle_floor(make_system, X0_fn, step_fn, nsteps):
    """Run the oracle (reference) and its FLOOR_VARIANTS; return (reference,
    per-field rounding floor = largest deviation of a variant)."""
    def run(cheb, lu):
        sysr = make_system(cheb, lu)
        X = X0_fn(sysr)
        st = step_fn(sysr)
        for _ in range(nsteps):
            X = st.step(X, st.dt)
        return X

    ref = run("mmt", "auto")
    floor = dict.fromkeys(NAMES, 0.0)
    for cheb, lu in FLOOR_VARIANTS:
        for k, v in field_errors(run(cheb, lu), ref, NAMES).items():
            floor[k] = max(floor[k], v)
    return ref, floor


def record(label, field, err, floor, bar):
    """Print one parity figure and append it (JSON line) to the file named by
    SPECTAU_PARITY_LOG when that is set: the measured error, the oracle
    variants' floor, and the bar the test applied."""
    line = {"test": label, "field": field, "err": float(err),
            "floor": None if floor is None else float(floor), "bar": float(bar)}
    print("parity", json.dumps(line))
    out = os.environ.get("SPECTAU_PARITY_LOG")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps(line) + "\n")


def check_fields(got, ref, floor, bar, label=None, names=None):
    names = names or NAMES
    errs = field_errors(got, ref, names)
    tol = {v: max(bar, 10 * floor[v]) for v in errs}
    if label:
        for v in errs:
            record(label, v, errs[v], floor[v], tol[v])
    bad = {v: (errs[v], tol[v]) for v in errs if errs[v] >= tol[v]}
    assert not bad, {"errors": errs, "floor": floor, "failing (err, tol)": bad}


NAMES = ("b", "p", "u", "w", "bz", "uz", "wz")
