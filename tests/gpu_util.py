"""Shared helpers for the GPU tests (no method arithmetic here)."""
import numpy as np


def rel_err(got, ref):
    """||got - ref||_2 / ||ref||_2, absolute when the reference norm < 1e-30."""
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(np.asarray(got) - np.asarray(ref))
    return d if nr < 1e-30 else d / nr


def field_errors(got, ref, names):
    return {v: rel_err(got[i], ref[i]) for i, v in enumerate(names)}
