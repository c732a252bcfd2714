"""GB300-native IMEX spectral-tau timestep (Fourier x Chebyshev, sm_103a).

The step -- dealiased spectral transforms, grid products and banded tau
pencil solves -- runs in the CUDA library ``libspectau.so`` behind the C ABI
of ``include/spectau.h``; this package is its thin Python binding plus the
host-side problem assembler.
"""
from .tau import BCAlternative, BCSlot, Equation, PencilProblem, Term  # noqa: F401
from . import rb  # noqa: F401


def build(force=False):
    from .build import build as _b
    return _b(force=force)


def __getattr__(name):
    if name in ("Context", "TauSolver", "RBSolver"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
