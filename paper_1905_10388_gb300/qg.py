"""Potential-vorticity inversion with a stratification profile: a linear
boundary value problem with a non-constant coefficient, for the C ABI.

On Fourier(x) x Chebyshev(z in [0, 1]), given the potential vorticity q,
the stream function psi solves (X = (psi, psiz))

    psiz_def:  dz(psi) - psiz = 0
    pv:        dx dx psi + dz(S(z) psiz) = q

with S(z) = 1/N^2(z) given by its Chebyshev coefficients (Sec. "Non-constant
coefficients": multiplication by S is a banded operator whose width is the
number of retained coefficients), rigid walls psiz(0) = psiz(1) = 0, and
psi(1) = 0 in place of psiz(1) = 0 in the k_x = 0 pencil.  Solved once per
pencil by the library's banded LU (Sec. "Linear boundary value solver").
Both variables carry boundary rows and are Dirichlet-recombined; every
pencil is real without phases.
"""
from .tau import BCAlternative, BCSlot, Equation, PencilProblem, Term

VARIABLES = ("psi", "psiz")


def qg_pencil_problem(strat):
    eqs = [
        Equation("psiz_def", L=[Term("psi", "dz", 1.0), Term("psiz", "I", -1.0)]),
        Equation("pv", L=[Term("psi", "I", lambda k: -k * k), Term("psiz", "nccdz", 1.0, ncc=list(strat))]),
    ]
    slots = [BCSlot([BCAlternative("psiz", "left")]),
             BCSlot([BCAlternative("psiz", "right", condition=lambda k: k != 0),
                     BCAlternative("psi", "right", condition=lambda k: k == 0)])]
    return PencilProblem(VARIABLES, eqs, slots, recombine=("psi", "psiz"), row_order=("pv", "psiz_def"))
