"""Rayleigh-Benard convection as a first-order tau problem for the C ABI.

Reading of the workload (the paper gives no equations for it): free-fall
units, kappa = (Ra Pr)^(-1/2), nu = (Ra/Pr)^(-1/2), z in [0, 1], with
X = (b, p, u, w, bz, uz, wz) and

    bz_def:  dz(b) - bz = 0
    uz_def:  dz(u) - uz = 0
    wz_def:  dz(w) - wz = 0
    b:       dt(b) - kappa (dx dx b + dz bz)          = -(u dx b + w bz)
    u:       dt(u) - nu (dx dx u + dz uz) + dx p      = -(u dx u + w uz)
    w:       dt(w) - nu (dx dx w + dz wz) + dz p - b  = -(u dx w + w wz)
    div:     dx u + wz = 0

    b(0) = 1, b(1) = 0, u(0) = u(1) = 0, w(0) = 0, and w(1) = 0 for k_x != 0
    or the pressure gauge p(1) = 0 for k_x = 0.

Real-ification: u and uz carry the phase i (u = i u~), and the uz_def and
u equations and the u boundary rows are multiplied by -i; every pencil
matrix is then real.  b, p, u, w are Dirichlet-recombined (they carry the
boundary conditions); bz, uz, wz are not (their operators stay narrower).
"""
import numpy as np

from .tau import BCAlternative, BCSlot, Equation, PencilProblem, Term

VARIABLES = ("b", "p", "u", "w", "bz", "uz", "wz")

# Slot order of the variables inside a mode block and order of the equation
# rows inside a mode block.  Chosen by searching the orderings for the
# smallest kl + ku of the interleaved, recombined pencil: kl = 7, ku = 22, so
# U after partial pivoting (kl + ku = 29 superdiagonals) fits one 32-lane
# window of the solve kernel.
SLOT_ORDER = ("bz", "uz", "u", "p", "w", "b", "wz")
ROW_ORDER = ("bz_def", "uz_def", "div", "u", "wz_def", "w", "b")

# advective terms: F[eq] += coef * op_a(var_a) * op_b(var_b), op in {ID, DX}
BILINEAR_TERMS = (
    ("b", -1.0, "ID", "u", "DX", "b"), ("b", -1.0, "ID", "w", "ID", "bz"),
    ("u", -1.0, "ID", "u", "DX", "u"), ("u", -1.0, "ID", "w", "ID", "uz"),
    ("w", -1.0, "ID", "u", "DX", "w"), ("w", -1.0, "ID", "w", "ID", "wz"),
)


def chebyshev_nodes(n, a=0.0, b=1.0):
    """Gauss-Chebyshev nodes mapped to [a, b], ascending (Sec. "Chebyshev basis")."""
    return a + (b - a) * (1.0 - np.cos(np.pi * (np.arange(n) + 0.5) / n)) / 2.0


def rb_pencil_problem(Ra, Pr=1.0, variables=SLOT_ORDER, row_order=ROW_ORDER):
    kappa = (Ra * Pr) ** -0.5
    nu = (Ra / Pr) ** -0.5
    eqs = [
        Equation("bz_def", L=[Term("b", "dz", 1.0), Term("bz", "I", -1.0)]),
        Equation("uz_def", L=[Term("u", "dz", 1.0), Term("uz", "I", -1.0)], phase=1),
        Equation("wz_def", L=[Term("w", "dz", 1.0), Term("wz", "I", -1.0)]),
        Equation("b", M=[Term("b", "I", 1.0)],
                 L=[Term("b", "I", lambda k: kappa * k * k), Term("bz", "dz", -kappa)]),
        Equation("u", M=[Term("u", "I", 1.0)],
                 L=[Term("u", "I", lambda k: nu * k * k), Term("uz", "dz", -nu),
                    Term("p", "I", lambda k: 1j * k)], phase=1),
        Equation("w", M=[Term("w", "I", 1.0)],
                 L=[Term("w", "I", lambda k: nu * k * k), Term("wz", "dz", -nu),
                    Term("p", "dz", 1.0), Term("b", "I", -1.0)]),
        Equation("div", L=[Term("u", "I", lambda k: 1j * k), Term("wz", "I", 1.0)]),
    ]
    order = {v: i for i, v in enumerate(variables)}
    eqs.sort(key=lambda e: order[{"bz_def": "bz", "uz_def": "uz", "wz_def": "wz",
                                  "b": "b", "u": "u", "w": "w", "div": "p"}[e.name]])
    slots = [
        BCSlot([BCAlternative("b", "left", value=lambda k: np.where(k == 0, 1.0, 0.0))]),
        BCSlot([BCAlternative("b", "right")]),
        BCSlot([BCAlternative("u", "left", phase=1)]),
        BCSlot([BCAlternative("u", "right", phase=1)]),
        BCSlot([BCAlternative("w", "left")]),
        BCSlot([BCAlternative("w", "right", condition=lambda k: k != 0),
                BCAlternative("p", "right", condition=lambda k: k == 0)]),
    ]
    return PencilProblem(variables, eqs, slots, recombine=("b", "p", "u", "w"),
                         var_phase={"u": 1, "uz": 1}, row_order=row_order)


def rb_onset_pencil_problem(Ra, Pr=1.0, variables=SLOT_ORDER, row_order=ROW_ORDER):
    """The linearization about the conductive state b = 1 - z (u = w = 0):
    the advection w dz(b0) = -w of the background moves to the b equation's
    left side as -w (eigenproblems: sigma M X + L X = 0)."""
    pr = rb_pencil_problem(Ra, Pr, variables, row_order)
    pr.eq_by_name["b"].L.append(Term("w", "I", -1.0))
    return pr


# --- three dimensions: Fourier x, Fourier y, Chebyshev z ----------------------

VARIABLES_3D = ("b", "p", "u", "v", "w", "bz", "uz", "vz", "wz")

# Slot and row orders of the 3D pencil (searched like the 2D ones).
SLOT_ORDER_3D = ("bz", "uz", "vz", "u", "v", "p", "w", "b", "wz")
ROW_ORDER_3D = ("bz_def", "uz_def", "vz_def", "div", "u", "v", "wz_def", "w", "b")

# advective terms with the y-derivative: F[eq] += coef * op_a(var_a) * op_b(var_b)
BILINEAR_TERMS_3D = tuple(
    (e, -1.0, "ID", a, op, f)
    for e in ("b", "u", "v", "w")
    for (a, op, f) in (("u", "DX", e), ("v", "DY", e), ("w", "ID", e + "z"))
)


def rb3d_pencil_problem(Ra, Pr=1.0, variables=SLOT_ORDER_3D, row_order=ROW_ORDER_3D):
    """3D Rayleigh-Benard, X = (b, p, u, v, w, bz, uz, vz, wz): the 2D system
    with v, vz, the v equation and dy terms; the wavenumber is (k_x, k_y).

    Real-ification: u, uz, v, vz carry the phase i and the uz_def, vz_def, u,
    v equations and the u, v boundary rows are multiplied by -i.
    """
    kappa = (Ra * Pr) ** -0.5
    nu = (Ra / Pr) ** -0.5
    k2 = lambda k: k[0] * k[0] + k[1] * k[1]
    eqs = [
        Equation("bz_def", L=[Term("b", "dz", 1.0), Term("bz", "I", -1.0)]),
        Equation("uz_def", L=[Term("u", "dz", 1.0), Term("uz", "I", -1.0)], phase=1),
        Equation("vz_def", L=[Term("v", "dz", 1.0), Term("vz", "I", -1.0)], phase=1),
        Equation("wz_def", L=[Term("w", "dz", 1.0), Term("wz", "I", -1.0)]),
        Equation("b", M=[Term("b", "I", 1.0)],
                 L=[Term("b", "I", lambda k: kappa * k2(k)), Term("bz", "dz", -kappa)]),
        Equation("u", M=[Term("u", "I", 1.0)],
                 L=[Term("u", "I", lambda k: nu * k2(k)), Term("uz", "dz", -nu),
                    Term("p", "I", lambda k: 1j * k[0])], phase=1),
        Equation("v", M=[Term("v", "I", 1.0)],
                 L=[Term("v", "I", lambda k: nu * k2(k)), Term("vz", "dz", -nu),
                    Term("p", "I", lambda k: 1j * k[1])], phase=1),
        Equation("w", M=[Term("w", "I", 1.0)],
                 L=[Term("w", "I", lambda k: nu * k2(k)), Term("wz", "dz", -nu),
                    Term("p", "dz", 1.0), Term("b", "I", -1.0)]),
        Equation("div", L=[Term("u", "I", lambda k: 1j * k[0]), Term("v", "I", lambda k: 1j * k[1]),
                           Term("wz", "I", 1.0)]),
    ]
    order = {v: i for i, v in enumerate(variables)}
    owner = {"bz_def": "bz", "uz_def": "uz", "vz_def": "vz", "wz_def": "wz", "b": "b", "u": "u", "v": "v",
             "w": "w", "div": "p"}
    eqs.sort(key=lambda e: order[owner[e.name]])
    zero = lambda k: (k[0] == 0) & (k[1] == 0)
    slots = [
        BCSlot([BCAlternative("b", "left", value=lambda k: np.where(zero(k), 1.0, 0.0))]),
        BCSlot([BCAlternative("b", "right")]),
        BCSlot([BCAlternative("u", "left", phase=1)]),
        BCSlot([BCAlternative("u", "right", phase=1)]),
        BCSlot([BCAlternative("v", "left", phase=1)]),
        BCSlot([BCAlternative("v", "right", phase=1)]),
        BCSlot([BCAlternative("w", "left")]),
        BCSlot([BCAlternative("w", "right", condition=lambda k: ~zero(k)),
                BCAlternative("p", "right", condition=zero)]),
    ]
    return PencilProblem(variables, eqs, slots, recombine=("b", "p", "u", "v", "w"),
                         var_phase={"u": 1, "uz": 1, "v": 1, "vz": 1}, row_order=row_order)
