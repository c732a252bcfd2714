"""Runge-Kutta IMEX step for problems with very many pencils (oracle; test
infrastructure, used only to write stored references).

The same step as ``timesteppers.RungeKuttaIMEX.step`` (Sec. "Runge-Kutta IMEX
integrators"): for stage i,

    B_p = M_p x0_p + dt sum_{j<i} A_ij F~_jp - dt sum_{j<i} H_ij L_p x_jp,
    x_ip = (M_p + dt H_ii L_p)^{-1} B_p,

with F~_j the left-preconditioned, boundary-filled right-hand side of the
stage-j state.  The per-pencil work is done where the pencil is solved: its
matrices, its factor (``timesteppers.PencilLU`` on that one pencil, the same
method choice) and the products M_p x0_p, L_p x_jp are built for the stage
and dropped afterwards, so no factor is held across pencils or stages (the
3D workload has 32768 pencils of 1152 unknowns; the plain step would keep
all their factors).  Every operation per pencil is the plain step's, in the
same order, so the two give identical results
(``tests/test_oracle_pencilwise.py``).  The pencil loop takes an optional
``map_fn`` (for example a process pool's ``map``) over chunks of pencils;
with a pool, ``problem_factory`` (a picklable callable returning the
system's pencil problem, e.g. ``functools.partial(problem_only,
rb3d.rb3d_problem, n_z, Ra, Pr)``) rebuilds the problem in each worker,
since the problem's coefficient functions do not pickle.
"""
import numpy as np

from .timesteppers import RK222, PencilLU


def problem_only(make, *args):
    """The problem of a constructor that returns (problem, ...)."""
    return make(*args)[0]


_WORKER_PROBLEMS = {}


def _stage_chunk(args):
    """Stage solves of a chunk of pencils (module level: picklable for pools)."""
    (src, wavenumbers, x0, xs, Fs, dt, A_row, H_row, i, method) = args
    if callable(src):
        key = repr(src)
        if key not in _WORKER_PROBLEMS:
            _WORKER_PROBLEMS[key] = src()
        problem = _WORKER_PROBLEMS[key]
    else:
        problem = src
    out = []
    for q, k in enumerate(wavenumbers):
        M, L = problem.pencil_matrices(k)
        B = (M @ x0[q]).copy()
        for j in range(i):
            if A_row[j] != 0.0:
                B = B + dt * A_row[j] * Fs[j][q]
            if H_row[j] != 0.0:
                B = B - dt * H_row[j] * (L @ xs[j][q])
        lu = PencilLU([(M, L)], 1.0, dt * H_row[i], method)
        out.append(lu.solve(0, B))
    return out


class RungeKuttaIMEXPencilwise:
    """``step(X0, dt)`` as RungeKuttaIMEX, pencil by pencil (see module doc)."""

    def __init__(self, system, tableau=RK222, map_fn=None, chunk=512, problem_factory=None):
        self.sys = system
        self.problem_src = problem_factory if problem_factory is not None else system.problem
        self.H, self.A = tableau["H"], tableau["A"]
        self.s = self.H.shape[0] - 1
        self.map_fn = map_fn or (lambda f, it: list(map(f, it)))
        self.chunk = int(chunk)

    def _wavenumber(self, p):
        s = self.sys
        return s.wavenumber(p) if hasattr(s, "wavenumber") else s.kx[p]

    def step(self, X0, dt):
        sys = self.sys
        P = sys.P
        method = getattr(sys, "lu_method", "auto")
        x0 = [sys.to_pencil(X0, p) for p in range(P)]
        xs, Fs = [], []
        X_prev = X0
        x_prev = x0
        for i in range(1, self.s + 1):
            Fs.append(sys.rhs_vectors(X_prev))
            xs.append(x_prev)
            jobs = []
            for p0 in range(0, P, self.chunk):
                p1 = min(P, p0 + self.chunk)
                jobs.append((self.problem_src, [self._wavenumber(p) for p in range(p0, p1)], x0[p0:p1],
                             [x[p0:p1] for x in xs], [F[p0:p1] for F in Fs], dt,
                             np.asarray(self.A[i]), np.asarray(self.H[i]), i, method))
            x_new = []
            for part in self.map_fn(_stage_chunk, jobs):
                x_new.extend(part)
            x_prev = x_new
            X_prev = sys.from_pencils(x_new)
        return X_prev
