"""Gradient of a final-state misfit through many steps (discrete adjoint).

Workload: J = 1/2 sum over the scale-1 grid of (b(T) - b_target)^2, control q
on the scale-1 grid entering the initial buoyancy as
b0 = 1 - z + (A xi + q) z (1 - z), bz0 = dz b0.  The forward sweep stores a
checkpoint of the state every ``checkpoint`` steps; the backward sweep
replays each segment from its checkpoint, recording every step's start and
stage states on the device (``sp_step_record``), and runs the adjoint steps
in reverse from those records (``sp_step_adjoint``).
Everything numeric runs in the library's kernels; torch holds device buffers
and the loss.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L
from . import rb as rbmod


class RBAdjoint:
    def __init__(self, solver, noise, target_grid, amplitude=1e-3, checkpoint=50):
        assert solver.scheme in ("RK222", "RK111"), "adjoint steps exist for the RK schemes"
        self.s = solver
        self.noise = np.asarray(noise, dtype=np.float64)
        self.target = torch.as_tensor(np.asarray(target_grid, dtype=np.float64), device="cuda")
        self.A = amplitude
        self.K = int(checkpoint)
        h = solver.ctx.handle
        L.check(h, L.lib().sp_adjoint_init(h, solver.pid))
        self.z = rbmod.chebyshev_nodes(solver.Nz)[:, None]
        self.shape = (solver.S, solver.P, solver.Nz)

    # -- device state helpers ------------------------------------------------
    def _get_state(self):
        s = self.s
        X = torch.empty(self.shape, dtype=torch.complex128, device="cuda")
        h = s.ctx.handle
        for i, v in enumerate(s.problem.variables):
            L.check(h, L.lib().sp_get_field(h, s.pid, s.var[v], ctypes.c_void_p(X[i].data_ptr()), 1, b"c"))
        return X

    def _set_state(self, X):
        s = self.s
        h = s.ctx.handle
        for i, v in enumerate(s.problem.variables):
            L.check(h, L.lib().sp_set_field(h, s.pid, s.var[v], ctypes.c_void_p(X[i].data_ptr()), 1, b"c"))

    def _set_initial(self, q):
        s = self.s
        b_grid = 1.0 - self.z + (self.A * self.noise + np.asarray(q, np.float64)) * self.z * (1.0 - self.z)
        zero = np.zeros((s.P, s.Nz), np.complex128)
        for v in s.problem.variables:
            s.set_field(v, zero)
        s.set_field("b", b_grid, layout="g")
        s.dz("b", "bz")

    # -- forward / backward ----------------------------------------------------
    def forward(self, q, nsteps):
        """Run nsteps; return the loss and the checkpoints (device states)."""
        s = self.s
        self._set_initial(q)
        checkpoints = []
        for n0 in range(0, nsteps, self.K):
            checkpoints.append(self._get_state())
            s.step(min(self.K, nsteps - n0))
        h = s.ctx.handle
        b = torch.empty((s.Nz, s.Nx), dtype=torch.float64, device="cuda")
        L.check(h, L.lib().sp_get_field(h, s.pid, s.var["b"], ctypes.c_void_p(b.data_ptr()), 1, b"g"))
        r = b - self.target
        J = 0.5 * float(torch.sum(r * r))
        return J, checkpoints, r

    def backward(self, checkpoints, r, nsteps):
        """dJ/dq from the residual r of the final buoyancy."""
        s = self.s
        h = s.ctx.handle
        lam = torch.zeros(self.shape, dtype=torch.complex128, device="cuda")
        rb = r.contiguous()
        # transpose of the scale-1 backward transform of b (lam is indexed by
        # the solver's variable slots)
        L.check(h, L.lib().sp_transform_adjoint(h, s.pid, ctypes.c_void_p(rb.data_ptr()),
                                                ctypes.c_void_p(lam[s.var["b"]].data_ptr()), 1, -1, 1, 1, 1))
        ns = 2 if s.scheme == "RK222" else 1                  # recorded states per step
        rec = torch.empty((min(self.K, max(nsteps, 1)), ns) + self.shape, dtype=torch.complex128, device="cuda")
        per_step = ns * int(np.prod(self.shape)) * 16
        for seg in reversed(range(len(checkpoints))):
            n0 = seg * self.K
            m = min(nsteps, n0 + self.K) - n0
            # replay the segment from its checkpoint, recording each step's states
            self._set_state(checkpoints[seg])
            L.check(h, L.lib().sp_step_record(h, s.pid, s.dt, m, ctypes.c_void_p(rec.data_ptr())))
            for k in reversed(range(m)):
                L.check(h, L.lib().sp_step_adjoint(h, s.pid, s.dt, ctypes.c_void_p(rec.data_ptr() + k * per_step),
                                                   ns, ctypes.c_void_p(lam.data_ptr())))
        # initial-state map: b coefficients from the grid, bz = dz b
        cb = lam[s.var["b"]].clone()
        L.check(h, L.lib().sp_dz_adjoint(h, s.pid, ctypes.c_void_p(lam[s.var["bz"]].data_ptr()),
                                         ctypes.c_void_p(cb.data_ptr())))
        g = torch.empty((s.Nz, s.Nx), dtype=torch.float64, device="cuda")
        L.check(h, L.lib().sp_transform_adjoint(h, s.pid, ctypes.c_void_p(cb.data_ptr()),
                                                ctypes.c_void_p(g.data_ptr()), 1, +1, 1, 1, 1))
        zz = torch.as_tensor(self.z * (1.0 - self.z), device="cuda")
        return g * zz

    def loss_and_grad(self, q, nsteps):
        J, cps, r = self.forward(q, nsteps)
        return J, self.backward(cps, r, nsteps)


class _RBLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, adj, nsteps):
        J, cps, r = adj.forward(q.detach().cpu().numpy(), nsteps)
        ctx.adj, ctx.cps, ctx.r, ctx.nsteps = adj, cps, r, nsteps
        return torch.tensor(J, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx, gJ):
        g = ctx.adj.backward(ctx.cps, ctx.r, ctx.nsteps)
        return (gJ * g).to(gJ.device), None, None


def rb_loss(q, adj, nsteps):
    """Differentiable loss J(q) of the adjoint workload (torch autograd)."""
    return _RBLoss.apply(q, adj, nsteps)
