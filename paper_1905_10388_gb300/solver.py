"""Thin Python front end over the C ABI: a pencil problem on one GPU.

``TauSolver`` hands an assembled :class:`~.tau.PencilProblem` to the library
(``sp_add_problem``, ``sp_set_layout``, ``sp_set_pencils``,
``sp_set_bilinear_rhs``) and exposes factor / step / state access.  Every
step of the method runs in the CUDA kernels behind the ABI; this module only
marshals arguments.  ``RBSolver`` builds the Rayleigh-Benard workload.
"""
import ctypes

import numpy as np

from . import _lib as L
from . import fisher as fkmod
from . import qg as qgmod
from . import rb as rbmod


class Context:
    """A library context on one CUDA device and stream."""

    def __init__(self, device=0, stream=None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        self._h = ctypes.c_void_p()
        st = L.lib().sp_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(stream))
        if st != L.SP_OK:
            raise L.SpectauError(st, "sp_create failed (is a CUDA device visible?)")
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            L.lib().sp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self):
        pen = ctypes.c_int64(-1)
        st = L.lib().sp_sync_status(self._h, ctypes.byref(pen))
        return st, pen.value


class TauSolver:
    """One Fourier(x) [x Fourier(y)] x Chebyshev(z) first-order problem in the
    library (``n_y`` given: three dimensions, pencil p = i_y N_x/2 + i_x)."""

    def __init__(self, ctx, problem, n_x, n_z, L_x, kx_scale=None, scheme="RK222",
                 precision="fp64", dealias=(3, 2), z_interval=(0.0, 1.0), bilinear=(), n_y=None, L_y=None):
        self.ctx = ctx
        self.problem = problem
        self.Nx, self.Nz, self.Lx = int(n_x), int(n_z), float(L_x)
        self.ndim = 2 if n_y is None else 3
        self.Ny = 1 if n_y is None else int(n_y)
        self.Ly = float(L_y) if L_y is not None else None
        self.K = self.Nx // 2
        self.P = self.Ny * self.K
        self.S = problem.S
        self.var = {v: i for i, v in enumerate(problem.variables)}
        self.state_order = tuple(problem.variables)   # order of get_state / set_state
        self.eq = {e.name: i for i, e in enumerate(problem.equations)}
        lib, h = L.lib(), ctx.handle
        bases = (L.sp_basis * self.ndim)()
        bases[0] = L.sp_basis(L.SP_FOURIER, self.Nx, 0.0, self.Lx, dealias[0], dealias[1])
        if self.ndim == 3:
            bases[1] = L.sp_basis(L.SP_FOURIER, self.Ny, 0.0, self.Ly, dealias[0], dealias[1])
        bases[self.ndim - 1] = L.sp_basis(L.SP_CHEBYSHEV, self.Nz, z_interval[0], z_interval[1],
                                          dealias[0], dealias[1])
        pid = ctypes.c_int()
        prec = L.SP_PREC_MIXED if precision == "mixed" else L.SP_PREC_FP64
        L.check(h, lib.sp_add_problem(h, self.ndim, bases, self.S, L.SCHEMES[scheme], prec, ctypes.byref(pid)))
        self.pid = pid.value
        self.scheme, self.precision = scheme, precision
        kx = 2 * np.pi * np.arange(self.K) / self.Lx
        if self.ndim == 2:
            wavenumbers = kx
        else:
            iy = np.arange(self.Ny)
            ky = 2 * np.pi * np.where(iy < self.Ny // 2, iy, iy - self.Ny) / self.Ly
            wavenumbers = (np.tile(kx, self.Ny), np.repeat(ky, self.K))
        asm = problem.build(self.Nz, wavenumbers, values=self.P <= 4096)
        self.assembly = asm
        c = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        bcv = np.ascontiguousarray(np.stack([asm["bc_values"].real, asm["bc_values"].imag], -1), dtype=np.float64)
        L.check(h, lib.sp_set_layout(h, self.pid, L.i32(c(asm["col_map"])), L.i32(c(asm["row_map"])),
                                     L.i32(c(asm["var_recombine"])), L.i32(c(asm["var_phase"])),
                                     L.i32(c(asm["eq_differential"])), L.i32(c(asm["eq_phase"])),
                                     len(asm["bc_rows"]), L.i32(c(asm["bc_rows"])), L.f64(bcv)))
        chunk = 4096                                   # pencils per sp_set_pencils call
        for p0 in range(0, self.P, chunk):
            p1 = min(self.P, p0 + chunk)
            Mv, Lv = asm["values"](p0, p1)
            L.check(h, lib.sp_set_pencils(h, self.pid, p0, p1 - p0, asm["n"], len(asm["indices"]),
                                          L.i32(c(asm["indptr"])), L.i32(c(asm["indices"])), L.f64(Mv), L.f64(Lv)))
        self.set_bilinear(bilinear)
        self.dt = None

    def set_solve_kernel(self, kind):
        """'auto', 'window', 'lanes' or 'spike' (before the problem moves to the device)."""
        h = self.ctx.handle
        L.check(h, L.lib().sp_set_solve_kernel(h, self.pid, L.SOLVE_KERNELS[kind]))

    def solve_lbvp(self, F):
        """Linear boundary value solve into the state: F maps equation name
        -> [P, N_z] complex T coefficients of its right-hand side."""
        names = list(F)
        eqs = np.array([self.eq[e] for e in names], np.int32)
        data = np.ascontiguousarray(np.stack([np.asarray(F[e], np.complex128) for e in names])) if names \
            else np.zeros((1, self.P, self.Nz), np.complex128)
        h = self.ctx.handle
        L.check(h, L.lib().sp_solve_lbvp(h, self.pid, len(names), L.i32(eqs), data.ctypes.data_as(ctypes.c_void_p)))
        return self.get_state()

    def set_z_transform(self, kind):
        """'auto', 'fft' or 'mma' (tensor cores; mixed precision; before the
        problem moves to the device)."""
        h = self.ctx.handle
        L.check(h, L.lib().sp_set_z_transform(h, self.pid, L.Z_TRANSFORMS[kind]))

    def z_transform(self):
        out = ctypes.c_int()
        h = self.ctx.handle
        L.check(h, L.lib().sp_get_z_transform(h, self.pid, ctypes.byref(out)))
        return {v: k for k, v in L.Z_TRANSFORMS.items()}[out.value]

    def set_spike_blocks(self, nblk):
        """Row blocks per pencil of the partitioned substitution (0: automatic)."""
        h = self.ctx.handle
        L.check(h, L.lib().sp_set_spike_blocks(h, self.pid, int(nblk)))

    def spike_blocks(self):
        """Row blocks per pencil in use (0: the substitution is not partitioned)."""
        out = ctypes.c_int()
        h = self.ctx.handle
        L.check(h, L.lib().sp_get_spike_blocks(h, self.pid, ctypes.byref(out)))
        return out.value

    def set_bilinear(self, terms):
        ops = {"ID": L.SP_OP_ID, "DX": L.SP_OP_DX, "DY": L.SP_OP_DY}
        eq = np.array([self.eq[t[0]] for t in terms], np.int32)
        coef = np.array([t[1] for t in terms], np.float64)
        oa = np.array([ops[t[2]] for t in terms], np.int32)
        va = np.array([self.var[t[3]] for t in terms], np.int32)
        ob = np.array([ops[t[4]] for t in terms], np.int32)
        vb = np.array([self.var[t[5]] for t in terms], np.int32)
        h = self.ctx.handle
        L.check(h, L.lib().sp_set_bilinear_rhs(h, self.pid, len(terms), L.i32(eq), L.f64(coef), L.i32(oa),
                                               L.i32(va), L.i32(ob), L.i32(vb)))
        self.nl_eqs = []
        for t in terms:
            if t[0] not in self.nl_eqs:
                self.nl_eqs.append(t[0])

    # -- numerics ------------------------------------------------------------
    def factor(self, dt):
        h = self.ctx.handle
        L.check(h, L.lib().sp_factor(h, self.pid, float(dt)))
        self.dt = float(dt)

    def step(self, nsteps=1, dt=None, graph=False):
        dt = self.dt if dt is None else float(dt)
        h = self.ctx.handle
        f = L.lib().sp_step_graph if graph else L.lib().sp_step
        L.check(h, f(h, self.pid, dt, int(nsteps)))

    def sync(self):
        st, pen = self.ctx.sync_status()
        if st != L.SP_OK:
            raise L.SpectauError(st, f"device status at pencil {pen}")

    def band(self):
        n, kl, ku = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        h = self.ctx.handle
        L.check(h, L.lib().sp_get_band(h, self.pid, ctypes.byref(n), ctypes.byref(kl), ctypes.byref(ku)))
        return n.value, kl.value, ku.value

    def cfl_frequency(self, velocities):
        """Largest sum_v |v| / dx_axis over the dealiased grid of the current
        state; velocities = ((variable, axis), ...), axis in 'x', 'y', 'z'."""
        axis = {"x": 0, "y": 1, "z": 2}
        n = len(velocities)
        vs = (ctypes.c_int * n)(*[self.var[v] for v, _ in velocities])
        ax = (ctypes.c_int * n)(*[axis[a] for _, a in velocities])
        f = ctypes.c_double()
        h = self.ctx.handle
        L.check(h, L.lib().sp_cfl_frequency(h, self.pid, n, vs, ax, ctypes.byref(f)))
        return f.value

    def eig_target(self, sigma_t, iters=60, x0=None):
        """Eigenvalue sigma of sigma M~ X~ + L~ X~ = 0 nearest the real target
        sigma_t in every pencil (shift-and-invert power iteration in the
        library); x0: complex [P][n] start vectors in solve-variable order.
        Replaces the step's factorization (factor again before stepping)."""
        re, im = np.zeros(self.P), np.zeros(self.P)
        h = self.ctx.handle
        xp = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.complex128)
            xp = x0.ctypes.data_as(ctypes.c_void_p)
        L.check(h, L.lib().sp_eig_target(h, self.pid, float(sigma_t), int(iters), xp,
                                         re.ctypes.data_as(ctypes.c_void_p), im.ctypes.data_as(ctypes.c_void_p)))
        self.dt = None
        return re + 1j * im

    def eig_residual(self):
        """Relative residual ||(L~ + sigma M~) x|| / (||L~ x|| + |sigma| ||M~ x||)
        of the last eigensolve's pair in every pencil."""
        out = np.zeros(self.P)
        h = self.ctx.handle
        L.check(h, L.lib().sp_eig_residual(h, self.pid, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def eig_targets(self, targets, iters=60):
        """Several modes per pencil: the eigenvalue nearest each target
        ([len(targets), P]) and the residual of each pair."""
        vals, res = [], []
        for t in targets:
            vals.append(self.eig_target(t, iters))
            res.append(self.eig_residual())
        return np.array(vals), np.array(res)

    def solve_work(self):
        """(multiply-adds per row and real right-hand side, factor bytes per
        pencil) of the substitution as the solve kernel performs it."""
        fma, nb = ctypes.c_double(), ctypes.c_double()
        h = self.ctx.handle
        L.check(h, L.lib().sp_get_solve_work(h, self.pid, ctypes.byref(fma), ctypes.byref(nb)))
        return fma.value, nb.value

    # -- state -----------------------------------------------------------------
    def set_field(self, name, data, layout="c"):
        h = self.ctx.handle
        if hasattr(data, "data_ptr"):        # a torch CUDA tensor
            L.check(h, L.lib().sp_set_field(h, self.pid, self.var[name], ctypes.c_void_p(data.data_ptr()), 1,
                                            layout.encode()))
            return
        arr = np.ascontiguousarray(data, dtype=np.complex128 if layout == "c" else np.float64)
        L.check(h, L.lib().sp_set_field(h, self.pid, self.var[name], arr.ctypes.data_as(ctypes.c_void_p), 0,
                                        layout.encode()))

    def get_field(self, name, layout="c"):
        h = self.ctx.handle
        if layout == "c":
            out = np.zeros((self.P, self.Nz), np.complex128)
        else:
            out = np.zeros(self.grid_shape(), np.float64)
        L.check(h, L.lib().sp_get_field(h, self.pid, self.var[name], out.ctypes.data_as(ctypes.c_void_p), 0,
                                        layout.encode()))
        return out

    def grid_shape(self, scale=(1, 1)):
        g = lambda n: n * scale[0] // scale[1]
        return (g(self.Nz), g(self.Nx)) if self.ndim == 2 else (g(self.Nz), g(self.Ny), g(self.Nx))

    def get_state(self):
        """State coefficients [var][p][m] in ``state_order``."""
        return np.stack([self.get_field(v) for v in self.state_order])

    def set_state(self, X):
        """Set every variable from X[var] (``state_order``)."""
        for i, v in enumerate(self.state_order):
            self.set_field(v, X[i])

    def dz(self, src, dst):
        h = self.ctx.handle
        L.check(h, L.lib().sp_dz(h, self.pid, self.var[src], self.var[dst]))

    def transform(self, data, direction, scale=(1, 1)):
        """direction -1: coefficients [f][p][m] -> grid [f][iz][ix] (3D:
        [f][iz][iy][ix]); +1: back."""
        h = self.ctx.handle
        if direction < 0:
            inp = np.ascontiguousarray(data, np.complex128)
            nf = inp.shape[0]
            out = np.zeros((nf,) + self.grid_shape(scale), np.float64)
        else:
            inp = np.ascontiguousarray(data, np.float64)
            nf = inp.shape[0]
            out = np.zeros((nf, self.P, self.Nz), np.complex128)
        L.check(h, L.lib().sp_transform(h, self.pid, inp.ctypes.data_as(ctypes.c_void_p),
                                        out.ctypes.data_as(ctypes.c_void_p), nf, int(direction),
                                        scale[0], scale[1], 0))
        return out

    def eval_rhs(self):
        out = np.zeros((max(1, len(self.nl_eqs)), self.P, self.Nz), np.complex128)
        ne = ctypes.c_int()
        h = self.ctx.handle
        L.check(h, L.lib().sp_eval_rhs(h, self.pid, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ne)))
        return {e: out[i] for i, e in enumerate(self.nl_eqs)}

    def set_timing(self, max_launches):
        h = self.ctx.handle
        L.check(h, L.lib().sp_set_timing(h, self.pid, int(max_launches)))

    def solve_time(self):
        ms, cnt = ctypes.c_double(), ctypes.c_int()
        h = self.ctx.handle
        L.check(h, L.lib().sp_last_solve_time(h, self.pid, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value


class CFL:
    """CFL timestep control (Sec. "Timestep determination") around a solver:
    the frequency of the current state from the library (sp_cfl_frequency),
    the step from the library's bounded, thresholded rule (sp_cfl_dt).
    ``step(n)`` advances n steps, choosing dt before each and factoring only
    when dt changes (the stored factorization is reused otherwise)."""

    def __init__(self, solver, velocities, initial_dt, safety=0.5, min_dt=0.0, max_dt=np.inf,
                 min_change=0.5, max_change=2.0, threshold=0.0):
        if not solver.scheme.startswith("RK"):
            raise ValueError("a changing step needs a Runge-Kutta scheme (SBDF here is constant-step)")
        self.solver, self.velocities = solver, tuple(velocities)
        self.dt = float(initial_dt)
        self.params = (float(safety), float(min_dt), float(max_dt), float(min_change), float(max_change),
                       float(threshold))
        self.history, self.factorizations = [], 0

    def compute_dt(self):
        freq = self.solver.cfl_frequency(self.velocities)
        out = ctypes.c_double()
        st = L.lib().sp_cfl_dt(freq, self.dt, *self.params, ctypes.byref(out))
        if st != 0:
            raise ValueError("inconsistent CFL bounds")
        self.dt = out.value
        return self.dt

    def step(self, nsteps=1):
        for _ in range(nsteps):
            dt = self.compute_dt()
            if self.solver.dt != dt:
                self.solver.factor(dt)
                self.factorizations += 1
            self.solver.step(1)
            self.history.append(dt)


class RBSolver(TauSolver):
    """2D Rayleigh-Benard convection (b, p, u, w, bz, uz, wz) in the library."""

    def __init__(self, ctx, n_x, n_z, Ra, Pr=1.0, L_x=4.0, scheme="RK222", precision="fp64",
                 dealias=(3, 2)):
        problem = rbmod.rb_pencil_problem(Ra, Pr)
        super().__init__(ctx, problem, n_x, n_z, L_x, scheme=scheme, precision=precision,
                         dealias=dealias, bilinear=rbmod.BILINEAR_TERMS)
        self.state_order = rbmod.VARIABLES
        self.Ra, self.Pr = Ra, Pr

    def set_initial_state(self, noise, amplitude=1e-3):
        """b = 1 - z + A xi z (1 - z) on the scale-1 grid (transformed on the
        device), bz = dz b (device recurrence), all other fields zero."""
        z = rbmod.chebyshev_nodes(self.Nz)[:, None]
        b_grid = 1.0 - z + amplitude * noise * z * (1.0 - z)
        zero = np.zeros((self.P, self.Nz), np.complex128)
        for v in self.problem.variables:
            self.set_field(v, zero)
        self.set_field("b", b_grid, layout="g")
        self.dz("b", "bz")


class FisherKPPSolver(TauSolver):
    """The Fisher-KPP example (u, uz) in the library: Fourier x on [0, L_x),
    Chebyshev z on [0, 1], Neumann walls."""

    def __init__(self, ctx, n_x, n_z, D=0.1, R=1.0, L_x=2 * np.pi, scheme="RK222", precision="fp64",
                 dealias=(3, 2)):
        problem = fkmod.fisher_pencil_problem(D, R)
        super().__init__(ctx, problem, n_x, n_z, L_x, scheme=scheme, precision=precision,
                         dealias=dealias, bilinear=fkmod.bilinear_terms(R))
        self.state_order = fkmod.VARIABLES
        self.D, self.R = D, R

    def set_initial_state(self, u_grid):
        """u from its values on the scale-1 grid [z, x] (transformed on the
        device), uz = dz u (device recurrence)."""
        self.set_field("u", np.asarray(u_grid, np.float64), layout="g")
        self.dz("u", "uz")


class RBOnsetEVP(TauSolver):
    """The linearization of 2D Rayleigh-Benard convection about the
    conductive state (b = 1 - z: the advection of the background adds -w to
    the b equation's L) as a pencil eigenproblem sigma M X + L X = 0; a
    perturbation grows as exp(sigma t), so sigma is the growth rate."""

    def __init__(self, ctx, n_x, n_z, Ra, Pr=1.0, L_x=4.0):
        super().__init__(ctx, rbmod.rb_onset_pencil_problem(Ra, Pr), n_x, n_z, L_x)
        self.state_order = rbmod.VARIABLES

    def growth_rates(self, target=0.0, iters=60, x0=None):
        """Growth rate sigma of the mode nearest `target` in every pencil."""
        return self.eig_target(target, iters, x0)


class QGInversion(TauSolver):
    """Potential-vorticity inversion dx dx psi + dz(S(z) dz psi) = q with the
    stratification S given by its Chebyshev coefficients (a linear boundary
    value problem with a non-constant coefficient)."""

    def __init__(self, ctx, n_x, n_z, strat, L_x=2 * np.pi, precision="fp64"):
        problem = qgmod.qg_pencil_problem(strat)
        super().__init__(ctx, problem, n_x, n_z, L_x, scheme="RK222", precision=precision)
        self.state_order = qgmod.VARIABLES

    def invert(self, q):
        """psi and psiz ([2, P, N_z] T coefficients) from q [P, N_z]."""
        return self.solve_lbvp({"pv": q})


class RB3DSolver(TauSolver):
    """3D Rayleigh-Benard convection (b, p, u, v, w, bz, uz, vz, wz) on
    Fourier x, Fourier y, Chebyshev z."""

    def __init__(self, ctx, n_x, n_y, n_z, Ra, Pr=1.0, L_x=4.0, L_y=4.0, scheme="RK222", precision="fp64",
                 dealias=(3, 2)):
        problem = rbmod.rb3d_pencil_problem(Ra, Pr)
        super().__init__(ctx, problem, n_x, n_z, L_x, scheme=scheme, precision=precision, dealias=dealias,
                         bilinear=rbmod.BILINEAR_TERMS_3D, n_y=n_y, L_y=L_y)
        self.state_order = rbmod.VARIABLES_3D
        self.Ra, self.Pr = Ra, Pr

    def set_initial_state(self, noise, amplitude=1e-3):
        """b = 1 - z + A xi z (1 - z) on the scale-1 grid (xi[z, y, x]), bz = dz b."""
        z = rbmod.chebyshev_nodes(self.Nz)[:, None, None]
        b_grid = 1.0 - z + amplitude * np.asarray(noise) * z * (1.0 - z)
        zero = np.zeros((self.P, self.Nz), np.complex128)
        for v in self.problem.variables:
            self.set_field(v, zero)
        self.set_field("b", b_grid, layout="g")
        self.dz("b", "bz")


def step_batched(solvers, nsteps=1, graph=True):
    """Advance several problems of one context together (``sp_step_batched``)."""
    ctx = solvers[0].ctx
    n = len(solvers)
    ids = (ctypes.c_int * n)(*[s.pid for s in solvers])
    dts = np.ascontiguousarray([s.dt for s in solvers], dtype=np.float64)
    L.check(ctx.handle, L.lib().sp_step_batched(ctx.handle, n, ids, L.f64(dts), int(nsteps), 1 if graph else 0))


def batch_tile(solvers):
    """z-kernel pencil tile chosen by the batch autotuner."""
    ctx = solvers[0].ctx
    n = len(solvers)
    ids = (ctypes.c_int * n)(*[s.pid for s in solvers])
    t = ctypes.c_int()
    L.check(ctx.handle, L.lib().sp_batch_tile(ctx.handle, n, ids, ctypes.byref(t)))
    return t.value


def batch_persistent(solvers):
    """True when the batch autotuner chose persistent grids for these solvers."""
    ctx = solvers[0].ctx
    n = len(solvers)
    ids = (ctypes.c_int * n)(*[s.pid for s in solvers])
    t = ctypes.c_int()
    L.check(ctx.handle, L.lib().sp_batch_persistent(ctx.handle, n, ids, ctypes.byref(t)))
    return bool(t.value)


def set_batch_persistent(solvers, mode):
    """Fix the batched launch shape: True (persistent grids), False (one CTA
    per work item) or None (the autotuner decides)."""
    ctx = solvers[0].ctx
    n = len(solvers)
    ids = (ctypes.c_int * n)(*[s.pid for s in solvers])
    m = -1 if mode is None else int(bool(mode))
    L.check(ctx.handle, L.lib().sp_set_batch_persistent(ctx.handle, n, ids, m))
