"""GPU discrete adjoint against the oracle adjoint and finite differences.

* one adjoint step (transposed stage solves, adjoint transforms and
  products) against oracle.adjoint.RBAdjoint.step_adjoint;
* the gradient of the final-buoyancy misfit through several steps, with
  checkpoint segments, against the oracle gradient and against central
  differences of the GPU forward loss (relative 1e-6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import rb as orb
from oracle.adjoint import RBAdjoint as OracleAdjoint
from oracle import timesteppers as ots
from paper_1905_10388_gb300 import _lib
from paper_1905_10388_gb300.adjoint import RBAdjoint, rb_loss
from paper_1905_10388_gb300.solver import Context, RBSolver

pytestmark = pytest.mark.gpu
NX, NZ, RA, DT = 16, 16, 1e5, 1e-2


def _to_slots(s, X_oracle):
    """Oracle variable order -> the solver's variable slots."""
    out = np.zeros_like(X_oracle)
    for i, v in enumerate(orb.RB_VARIABLES):
        out[s.var[v]] = X_oracle[i]
    return out


def _from_slots(s, X):
    return np.stack([X[s.var[v]] for v in orb.RB_VARIABLES])


def _ip(a, b):
    return float(np.real(np.sum(np.conj(a) * b)))


def test_transform_and_dz_adjoints_are_transposes():
    """<g, B c> = <B^T g, c>, <c, F g> = <F^T c, g>, <d, D c> = <D^T d, c>
    for the scale-1 transforms B (coefficients -> grid), F (grid ->
    coefficients) and the Chebyshev derivative D, each against its own
    forward entry point."""
    ctx = Context(0)
    s = RBSolver(ctx, 24, 16, 1e5, dealias=(2, 1))
    h, L = ctx.handle, _lib.lib()
    rng = np.random.default_rng(4)
    c = rng.standard_normal((2, s.P, s.Nz)) + 1j * rng.standard_normal((2, s.P, s.Nz))
    c[:, 0, :] = c[:, 0, :].real
    g = rng.standard_normal((2, s.Nz, s.Nx))
    Bc, Fg = s.transform(c, -1), s.transform(g, +1)
    gd = torch.as_tensor(g, device="cuda").contiguous()
    cd = torch.as_tensor(c, device="cuda").contiguous()
    BTg, FTc = torch.zeros_like(cd), torch.zeros_like(gd)
    _lib.check(h, L.sp_transform_adjoint(h, s.pid, gd.data_ptr(), BTg.data_ptr(), 2, -1, 1, 1, 1))
    _lib.check(h, L.sp_transform_adjoint(h, s.pid, cd.data_ptr(), FTc.data_ptr(), 2, +1, 1, 1, 1))
    a, b = _ip(g, Bc), _ip(BTg.cpu().numpy(), c)
    assert abs(a - b) < 1e-12 * abs(a), (a, b)
    a, b = _ip(c, Fg), _ip(FTc.cpu().numpy(), g)
    assert abs(a - b) < 1e-12 * abs(a), (a, b)
    cb = rng.standard_normal((s.P, s.Nz)) + 1j * rng.standard_normal((s.P, s.Nz))
    s.set_field("b", cb)
    s.dz("b", "bz")
    dbar = rng.standard_normal((s.P, s.Nz)) + 1j * rng.standard_normal((s.P, s.Nz))
    dd = torch.as_tensor(dbar, device="cuda").contiguous()
    cbar = torch.zeros_like(dd)
    _lib.check(h, L.sp_dz_adjoint(h, s.pid, dd.data_ptr(), cbar.data_ptr()))
    a, b = _ip(dbar, s.get_field("bz")), _ip(cbar.cpu().numpy(), cb)
    assert abs(a - b) < 1e-12 * abs(a), (a, b)
    ctx.close()


def test_step_adjoint_against_gpu_forward_differences():
    """<lam, dPhi(X0) V> by central differences of the GPU step equals
    <Phi'(X0)^H lam, V> from sp_step_adjoint (no oracle involved)."""
    ctx = Context(0)
    s = RBSolver(ctx, NX, NZ, RA, scheme="RK222")
    s.factor(DT)
    RBAdjoint(s, si.rb_noise(1, NZ, NX), np.zeros((NZ, NX)))
    s.set_initial_state(si.rb_noise(3, NZ, NX) * 50.0)
    s.step(2)
    X0 = s.get_state()
    rng = np.random.default_rng(21)
    lam = rng.standard_normal(X0.shape) + 1j * rng.standard_normal(X0.shape)
    V = rng.standard_normal(X0.shape) + 1j * rng.standard_normal(X0.shape)

    def phi(X):
        s.set_state(X)
        s.step(1)
        return s.get_state()

    def central(eps):
        return (_ip(lam, phi(X0 + eps * V)) - _ip(lam, phi(X0 - eps * V))) / (2 * eps)

    fd = (4 * central(5e-5) - central(1e-4)) / 3        # Richardson: O(eps^4)
    Xd = torch.as_tensor(_to_slots(s, X0), device="cuda").contiguous()
    Ld = torch.as_tensor(_to_slots(s, lam), device="cuda").contiguous()
    h = ctx.handle
    _lib.check(h, _lib.lib().sp_step_adjoint(h, s.pid, DT, Xd.data_ptr(), 1, Ld.data_ptr()))
    ctx.sync_status()
    an = _ip(_from_slots(s, Ld.cpu().numpy()), V)
    assert abs(fd - an) < 1e-8 * abs(fd), (fd, an)
    ctx.close()


@pytest.mark.parametrize("given_stage", [False, True])
def test_step_adjoint_matches_oracle(given_stage):
    """One adjoint step against the oracle, with the first stage recomputed
    from X^n (nstates = 1) or supplied (nstates = 2, the oracle's X^1)."""
    ctx = Context(0)
    s = RBSolver(ctx, NX, NZ, RA, scheme="RK222")
    s.factor(DT)
    RBAdjoint(s, si.rb_noise(1, NZ, NX), np.zeros((NZ, NX)))
    sysr = orb.RB2D(NX, NZ, RA)
    oadj = OracleAdjoint(sysr)
    X0 = oadj.initial_state_q(si.rb_noise(2, NZ, NX) * 50.0, 0.0)
    st = ots.RungeKuttaIMEX(sysr)
    for _ in range(3):
        X0 = st.step(X0, DT)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal(X0.shape) + 1j * rng.standard_normal(X0.shape)
    X1 = oadj.stage1(X0, DT)
    ref = oadj.step_adjoint(X0, X1, lam, DT)
    states = [_to_slots(s, X0)] + ([_to_slots(s, X1)] if given_stage else [])
    Xd = torch.as_tensor(np.stack(states), device="cuda").contiguous()
    Ld = torch.as_tensor(_to_slots(s, lam), device="cuda").contiguous()
    h = ctx.handle
    _lib.check(h, _lib.lib().sp_step_adjoint(h, s.pid, DT, Xd.data_ptr(), len(states), Ld.data_ptr()))
    ctx.sync_status()
    got = _from_slots(s, Ld.cpu().numpy())
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-10, err
    with pytest.raises(_lib.SpectauError):
        _lib.check(h, _lib.lib().sp_step_adjoint(h, s.pid, DT, Xd.data_ptr(), 3, Ld.data_ptr()))
    ctx.close()


def test_step_record_states():
    """sp_step_record advances like sp_step and records X^n and the stage
    state X^1 of every step (checked against the oracle's stage state)."""
    ctx = Context(0)
    a = RBSolver(ctx, NX, NZ, RA, scheme="RK222")
    b = RBSolver(ctx, NX, NZ, RA, scheme="RK222")
    for s in (a, b):
        s.factor(DT)
        s.set_initial_state(si.rb_noise(8, NZ, NX) * 50.0)
    a.step(3)
    rec = torch.zeros((3, 2, a.S, a.P, a.Nz), dtype=torch.complex128, device="cuda")
    h = ctx.handle
    _lib.check(h, _lib.lib().sp_step_record(h, b.pid, DT, 3, rec.data_ptr()))
    assert np.array_equal(a.get_state(), b.get_state())
    rec = rec.cpu().numpy()
    oadj = OracleAdjoint(orb.RB2D(NX, NZ, RA))
    for k in range(3):
        Xn, X1 = _from_slots(b, rec[k, 0]), _from_slots(b, rec[k, 1])
        ref = oadj.stage1(Xn, DT)
        assert np.linalg.norm(X1 - ref) < 1e-12 * np.linalg.norm(ref)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_gradient_matches_oracle_with_checkpoints(prec, tol):
    ctx = Context(0)
    s = RBSolver(ctx, NX, NZ, RA, scheme="RK222", precision=prec)
    s.factor(DT)
    noise = si.rb_noise(5, NZ, NX) * 50.0
    sysr = orb.RB2D(NX, NZ, RA)
    oadj = OracleAdjoint(sysr)
    target = sysr.to_grid(oadj.initial_state_q(si.rb_noise(6, NZ, NX) * 50.0, 0.0)[0], NX, NZ)
    q = 0.01 * np.random.default_rng(3).standard_normal((NZ, NX))
    nsteps = 7
    adj = RBAdjoint(s, noise, target, checkpoint=3)          # three segments
    J, g = adj.loss_and_grad(q, nsteps)
    Jr, gr = oadj.loss_and_grad(noise, target, q, DT, nsteps)
    assert abs(J - Jr) < tol * abs(Jr)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) < tol
    ctx.close()


def test_gradient_against_central_differences_and_autograd():
    ctx = Context(0)
    s = RBSolver(ctx, NX, NZ, RA, scheme="RK222")
    s.factor(DT)
    noise = si.rb_noise(7, NZ, NX) * 50.0
    target = np.zeros((NZ, NX))
    adj = RBAdjoint(s, noise, target, checkpoint=4)
    rng = np.random.default_rng(11)
    q = 0.01 * rng.standard_normal((NZ, NX))
    nsteps = 6
    qt = torch.tensor(q, device="cuda", requires_grad=True)
    J = rb_loss(qt, adj, nsteps)
    J.backward()
    g = qt.grad.cpu().numpy()
    for _ in range(2):
        d = rng.standard_normal((NZ, NX))
        eps = 1e-4
        Jp, _, _ = adj.forward(q + eps * d, nsteps)
        Jm, _, _ = adj.forward(q - eps * d, nsteps)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) < 1e-6 * abs(fd), (fd, an)
    ctx.close()


def test_gradient_repeats_bit_for_bit_on_the_partitioned_solve():
    """At 32 x 128 (896 rows per pencil) the forward and transposed solves
    take the partitioned back substitution, whose blocks start from the
    previous solve's inflows; setting the state resets those guesses, so a
    second gradient from the same state repeats the first exactly."""
    ctx = Context(0)
    nx, nz = 32, 128
    s = RBSolver(ctx, nx, nz, 1e6, scheme="RK222")
    s.factor(1e-3)
    assert s.spike_blocks() > 0
    noise = si.rb_noise(9, nz, nx) * 50.0
    adj = RBAdjoint(s, noise, np.zeros((nz, nx)), checkpoint=3)
    q = 0.01 * np.random.default_rng(12).standard_normal((nz, nx))
    J1, g1 = adj.loss_and_grad(q, 7)
    J2, g2 = adj.loss_and_grad(q, 7)
    assert J1 == J2
    assert np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())
    ctx.close()
