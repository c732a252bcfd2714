"""Fisher-KPP reaction-diffusion as a first-order tau problem for the C ABI.

The overview example of Sec. "Codebase structure": u(x, z, t) on a channel
periodic in x and bounded in z in [0, 1], X = (u, uz),

    uz_def:  dz(u) - uz = 0
    u:       dt(u) - D (dx dx u + dz uz) - R u = -R u u

with Neumann walls uz(0) = uz(1) = 0.  The reaction's linear part R u is
implicit (in L), its quadratic part the explicit bilinear right-hand side.
uz carries the boundary rows and is Dirichlet-recombined; every pencil is
real without phases.
"""
import numpy as np

from .tau import BCAlternative, BCSlot, Equation, PencilProblem, Term

VARIABLES = ("u", "uz")

# slot and row orders inside a mode block: the smallest kl + ku of the four
# (kl = 2, ku = 6)
SLOT_ORDER = ("u", "uz")
ROW_ORDER = ("u", "uz_def")


def fisher_pencil_problem(D, R, variables=SLOT_ORDER, row_order=ROW_ORDER):
    eqs = [
        Equation("uz_def", L=[Term("u", "dz", 1.0), Term("uz", "I", -1.0)]),
        Equation("u", M=[Term("u", "I", 1.0)],
                 L=[Term("u", "I", lambda k: D * k * k - R), Term("uz", "dz", -D)]),
    ]
    order = {v: i for i, v in enumerate(variables)}
    eqs.sort(key=lambda e: order[{"uz_def": "uz", "u": "u"}[e.name]])
    slots = [BCSlot([BCAlternative("uz", "left")]), BCSlot([BCAlternative("uz", "right")])]
    return PencilProblem(variables, eqs, slots, recombine=("uz",), row_order=row_order)


def bilinear_terms(R):
    """-R u u for the u equation."""
    return (("u", -float(R), "ID", "u", "ID", "u"),)
