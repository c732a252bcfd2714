"""IMEX timesteppers on pencil systems (oracle; test infrastructure only).

Restates Sec. "Timesteppers":

Multistep IMEX (Sec. "Multistep IMEX integrators"):
    (a_0 M + b_0 L) X^n = sum_{j=1..s} c_j F^{n-j} - a_j M X^{n-j} - b_j L X^{n-j}
with the first iterations taken at lower order.  The coefficients are the
semi-implicit BDF schemes of Wang & Ruuth (2008), cited by the paper but not
printed there; for a constant step:
    SBDF1: a = (1, -1)/dt,                   b = (1, 0, ...),  c = (-, 1)
    SBDF2: a = (3/2, -2, 1/2)/dt,            c = (-, 2, -1)
    SBDF3: a = (11/6, -3, 3/2, -1/3)/dt,     c = (-, 3, -3, 1)
    SBDF4: a = (25/12, -4, 3, -4/3, 1/4)/dt, c = (-, 4, -6, 4, -1)
(the backward-difference weights of the implicit part and the polynomial
extrapolation weights of the explicit part).  The Crank-Nicolson
Adams-Bashforth schemes of the same family (also cited, not printed):
    CNAB1: a = (1, -1)/dt,     b = (1/2, 1/2),     c = (-, 1)
    CNAB2: a = (1, -1, 0)/dt,  b = (1/2, 1/2, 0),  c = (-, 3/2, -1/2)
(the trapezoidal rule on the implicit part, Adams-Bashforth extrapolation
of the explicit part; CNAB2 starts with one CNAB1 step, and both orders
factor the same matrix M/dt + L/2).

Runge-Kutta IMEX (Sec. "Runge-Kutta IMEX integrators"):
    (M + dt H_ii L) X^i = M X^0 + dt sum_{j<i} A_ij F^j - dt sum_{j<i} H_ij L X^j
with X^{n+1} = X^s (globally stiffly accurate).  RK222 is the ARS(2,2,2)
scheme of Ascher, Ruuth & Spiteri (1997), cited but not printed:
    gamma = 1 - 1/sqrt(2), delta = 1 - 1/(2 gamma)
    H = [[0,0,0],[0,gamma,0],[0,1-gamma,gamma]]
    A = [[0,0,0],[gamma,0,0],[delta,1-delta,0]],  c = [0, gamma, 1]
RK111 (first order, one stage): H = [[0,0],[0,1]], A = [[0,0],[1,0]].
RK443 is the third-order, four-stage ARS(4,4,3) scheme of the same paper
(the method of the paper's MHD and annulus examples), also not printed
there: implicit diagonal 1/2 throughout, c = [0, 1/2, 2/3, 1/2, 1],
    H rows 1-4: [0,1/2], [0,1/6,1/2], [0,-1/2,1/2,1/2], [0,3/2,-3/2,1/2,1/2]
    A rows 1-4: [1/2], [11/18,1/18], [5/6,-5/6,1/2], [1/4,7/4,3/4,-7/4]

Pins: ``tests/test_oracle_timesteppers.py`` (amplification factors of the
linear test equation, exact decay of polynomial diffusion modes, second-order
convergence, SBDF two-term recurrence, the Crank-Nicolson factor of CNAB on a
polynomial mode and CNAB2's second order; for RK443 the third-order conditions
of both tableaux and of their coupling, third-order convergence of a
diffusion mode and of a stiff-linear / quadratic-explicit scalar problem with
a closed-form solution).

A "system" provides: P (pencil count), matrices() -> [(M_p, L_p)],
rhs_vectors(X) -> [F~_p], to_pencil(X, p), from_pencils(vectors).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

GAMMA = 1.0 - 1.0 / np.sqrt(2.0)
DELTA = 1.0 - 1.0 / (2.0 * GAMMA)

RK222 = dict(
    H=np.array([[0, 0, 0], [0, GAMMA, 0], [0, 1 - GAMMA, GAMMA]], dtype=np.float64),
    A=np.array([[0, 0, 0], [GAMMA, 0, 0], [DELTA, 1 - DELTA, 0]], dtype=np.float64),
    c=np.array([0.0, GAMMA, 1.0]),
)

RK111 = dict(
    H=np.array([[0, 0], [0, 1]], dtype=np.float64),
    A=np.array([[0, 0], [1, 0]], dtype=np.float64),
    c=np.array([0.0, 1.0]),
)

RK443 = dict(
    H=np.array([[0, 0, 0, 0, 0],
                [0, 1 / 2, 0, 0, 0],
                [0, 1 / 6, 1 / 2, 0, 0],
                [0, -1 / 2, 1 / 2, 1 / 2, 0],
                [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2]], dtype=np.float64),
    A=np.array([[0, 0, 0, 0, 0],
                [1 / 2, 0, 0, 0, 0],
                [11 / 18, 1 / 18, 0, 0, 0],
                [5 / 6, -5 / 6, 1 / 2, 0, 0],
                [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0]], dtype=np.float64),
    c=np.array([0.0, 1 / 2, 2 / 3, 1 / 2, 1.0]),
)

DENSE_LIMIT = 1000


class PencilLU:
    """LU factors of a*M_p + b*L_p for every pencil.

    method "auto": dense LAPACK getrf up to DENSE_LIMIT rows, else SuperLU
    with COLAMD column ordering; "natural": SuperLU in the natural column
    order (partial pivoting, the elimination order of a band solver);
    "dense": dense LAPACK getrf at any size.  All solve the same systems; the
    others give other rounding orders for floor estimates.
    """

    def __init__(self, mats, a, b, method="auto"):
        self.factors = []
        for (M, L) in mats:
            A = (a * M + b * L)
            if method == "natural":
                self.factors.append(("sparse", spla.splu(sps.csc_matrix(A), permc_spec="NATURAL")))
            elif method == "dense" or A.shape[0] <= DENSE_LIMIT:
                self.factors.append(("dense", sla.lu_factor(A.toarray())))
            else:
                self.factors.append(("sparse", spla.splu(sps.csc_matrix(A))))

    def solve(self, p, rhs):
        kind, f = self.factors[p]
        if kind == "dense":
            return sla.lu_solve(f, rhs)
        return f.solve(rhs)


class _Factors:
    def __init__(self, system):
        self.system = system
        self.cache = {}

    def get(self, a, b):
        key = (float(a), float(b))
        if key not in self.cache:
            self.cache[key] = PencilLU(self.system.matrices(), a, b,
                                       getattr(self.system, "lu_method", "auto"))
        return self.cache[key]


class RungeKuttaIMEX:
    def __init__(self, system, tableau=RK222):
        self.sys = system
        self.H, self.A = tableau["H"], tableau["A"]
        self.s = self.H.shape[0] - 1
        self.factors = _Factors(system)

    def step(self, X0, dt):
        sys = self.sys
        mats = sys.matrices()
        P = sys.P
        x0 = [sys.to_pencil(X0, p) for p in range(P)]
        MX0 = [mats[p][0] @ x0[p] for p in range(P)]
        F, LX = [], []
        X_prev = X0
        x_prev = x0
        for i in range(1, self.s + 1):
            F.append(sys.rhs_vectors(X_prev))
            LX.append([mats[p][1] @ x_prev[p] for p in range(P)])
            lu = self.factors.get(1.0, dt * self.H[i, i])
            x_new = []
            for p in range(P):
                B = MX0[p].copy()
                for j in range(i):
                    if self.A[i, j] != 0.0:
                        B = B + dt * self.A[i, j] * F[j][p]
                    if self.H[i, j] != 0.0:
                        B = B - dt * self.H[i, j] * LX[j][p]
                x_new.append(lu.solve(p, B))
            x_prev = x_new
            X_prev = sys.from_pencils(x_new)
        return X_prev


class SBDF:
    """SBDF1 .. SBDF4 multistep IMEX with the paper's general coefficient form;
    the first steps at the orders the history allows."""

    def __init__(self, system, order=2):
        self.sys = system
        self.order = int(order)
        self.factors = _Factors(system)
        self.hist_MX, self.hist_LX, self.hist_F = [], [], []  # newest first
        self.iteration = 0

    @staticmethod
    def coefficients(order, dt):
        if order == 1:
            return np.array([1.0, -1.0]) / dt, np.array([1.0, 0.0]), np.array([0.0, 1.0])
        if order == 2:
            return (np.array([1.5, -2.0, 0.5]) / dt, np.array([1.0, 0.0, 0.0]),
                    np.array([0.0, 2.0, -1.0]))
        if order == 3:
            return (np.array([11 / 6, -3.0, 3 / 2, -1 / 3]) / dt, np.array([1.0, 0.0, 0.0, 0.0]),
                    np.array([0.0, 3.0, -3.0, 1.0]))
        if order == 4:
            return (np.array([25 / 12, -4.0, 3.0, -4 / 3, 1 / 4]) / dt, np.array([1.0, 0.0, 0.0, 0.0, 0.0]),
                    np.array([0.0, 4.0, -6.0, 4.0, -1.0]))
        raise ValueError("order")

    def step(self, X, dt):
        sys = self.sys
        mats = sys.matrices()
        P = sys.P
        x = [sys.to_pencil(X, p) for p in range(P)]
        self.hist_MX.insert(0, [mats[p][0] @ x[p] for p in range(P)])
        self.hist_LX.insert(0, [mats[p][1] @ x[p] for p in range(P)])
        self.hist_F.insert(0, sys.rhs_vectors(X))
        order = min(self.order, self.iteration + 1)
        a, b, c = self.coefficients(order, dt)
        lu = self.factors.get(a[0], b[0])
        x_new = []
        for p in range(P):
            B = np.zeros_like(x[p])
            for j in range(1, order + 1):
                B = B + c[j] * self.hist_F[j - 1][p]
                B = B - a[j] * self.hist_MX[j - 1][p]
                B = B - b[j] * self.hist_LX[j - 1][p]
            x_new.append(lu.solve(p, B))
        keep = self.order
        del self.hist_MX[keep:], self.hist_LX[keep:], self.hist_F[keep:]
        self.iteration += 1
        return sys.from_pencils(x_new)


class CNAB(SBDF):
    """CNAB1 / CNAB2 (Crank-Nicolson Adams-Bashforth, Wang & Ruuth 2008),
    constant step, through the multistep form of ``SBDF.step``: the first
    step at first order."""

    @staticmethod
    def coefficients(order, dt):
        if order == 1:
            return np.array([1.0, -1.0]) / dt, np.array([0.5, 0.5]), np.array([0.0, 1.0])
        if order == 2:
            return (np.array([1.0, -1.0, 0.0]) / dt, np.array([0.5, 0.5, 0.0]),
                    np.array([0.0, 1.5, -0.5]))
        raise ValueError("order")
