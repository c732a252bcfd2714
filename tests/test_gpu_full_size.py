"""GPU parity at the workloads' stated sizes and lengths, against stored FP64
oracle references (``tests/golden/ref_*.npz``, written by
``tests/golden/make_references.py`` from ``oracle/`` alone).

* 2D Rayleigh-Benard 512 x 256, Ra = 1e8, SBDF2, dt = 1e-4: the state after
  1000 steps, FP64 and mixed;
* 3D Rayleigh-Benard 256 x 256 x 128, Ra = 1e7, RK222, dt = 5e-4: one step
  through the kernels the library picks at this size (lane substitution),
  mixed and FP64, on 64 sampled pencils;
* the 64-instance uneven batch advanced together (one launch per kernel type
  per stage, CUDA graph), RK222, 5 steps, four instances of it at their real
  sizes (512 x 256, 256 x 256, 64 x 256, 512 x 64);
* the gradient of the final-buoyancy misfit through 500 RK222 steps at
  256 x 128 with checkpoints every 50 steps, FP64 and mixed.

States are compared on a fixed seeded sample of their coefficients (the
references store that sample): per field ||x_gpu - x_ref|| / ||x_ref|| over
the sample.  Bars: FP64 max(1e-12, 10 x the floor), the floor being the
deviation of an oracle variant that sums the same arithmetic in another
order; mixed 1e-5 per field.  Every figure is printed and recorded.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from paper_1905_10388_gb300.adjoint import RBAdjoint
from paper_1905_10388_gb300.solver import Context, RB3DSolver, RBSolver, step_batched
from gpu_util import record, rel_err

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BAR = {"fp64": 1e-12, "mixed": 1e-5}


def _ref(name):
    p = os.path.join(GOLDEN, f"ref_{name}.npz")
    assert os.path.exists(p), f"stored reference {p} missing (tests/golden/make_references.py writes it)"
    return np.load(p)


def _check(label, got, ref, floor, names, prec):
    bad = {}
    for i, v in enumerate(names):
        err = rel_err(got[i], ref[i])
        tol = max(BAR[prec], 10 * float(floor[i])) if prec == "fp64" else BAR[prec]
        record(label, str(v), err, float(floor[i]), tol)
        if not err < tol:
            bad[str(v)] = (err, tol)
    assert not bad, bad


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rb2d_512x256_sbdf2_1000_steps(ctx, prec):
    R = _ref("rb2d_512x256_sbdf2_1000")
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="SBDF2", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(si.rb_noise(w.seed, w.n_z, w.n_x))
    s.step(int(R["steps"]), graph=True)
    ctx.sync_status()
    X = s.get_state()
    got = X.reshape(X.shape[0], -1)[:, R["flat"]]
    _check(f"rb2d_512x256_sbdf2_{prec}_1000steps", got, R["ref"], R["floor"], R["names"], prec)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_rb3d_256x256x128_rk222_one_step(ctx, prec):
    R = _ref("rb3d_256x256x128_rk222_1")
    w = si.WORKLOADS["rb3d_256x256x128_rk222"]
    s = RB3DSolver(ctx, w.n_x, w.n_y, w.n_z, w.Ra, w.Pr, w.L_x, w.L_y, scheme="RK222", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(si.rb_noise3(w.seed, w.n_z, w.n_y, w.n_x))
    s.step(1)
    ctx.sync_status()
    got = s.get_state()[:, R["pencils"], :]
    _check(f"rb3d_256x256x128_rk222_{prec}_1step_lanes", got, R["ref"], R["floor"], R["names"], prec)
    del s
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch64_instances_at_their_sizes(ctx, prec):
    R = _ref("batch64_rk222_5")
    ws = si.batched_workloads()
    solvers = []
    for w in ws:
        s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK222", precision=prec)
        s.factor(w.dt)
        s.set_initial_state(si.rb_noise(w.seed, w.n_z, w.n_x))
        solvers.append(s)
    step_batched(solvers, int(R["steps"]), graph=True)
    ctx.sync_status()
    for i in R["picks"]:
        X = solvers[int(i)].get_state()
        got = X.reshape(X.shape[0], -1)[:, R[f"flat_{i}"]]
        w = ws[int(i)]
        _check(f"batch64_instance{i}_{w.n_x}x{w.n_z}_rk222_{prec}_5steps", got, R[f"ref_{i}"], R[f"floor_{i}"],
               R["names"], prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_gradient_500_steps_checkpoint_50(ctx, prec):
    R = _ref("rb2d_256x128_adjoint_500")
    w = si.WORKLOADS["rb2d_256x128_rk222_adjoint"]
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK222", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(si.rb_noise(w.seed + 1, w.n_z, w.n_x))
    target = s.get_field("b", "g")                 # b*: the initial buoyancy of seed + 1
    adj = RBAdjoint(s, si.rb_noise(w.seed, w.n_z, w.n_x), target, checkpoint=int(R["checkpoint"]))
    J, g = adj.loss_and_grad(np.zeros((w.n_z, w.n_x)), int(R["steps"]))
    g = g.cpu().numpy()
    err = rel_err(g, R["grad"])
    floor = float(R["floor"])
    tol = max(BAR[prec], 10 * floor) if prec == "fp64" else BAR[prec]
    record(f"rb2d_256x128_adjoint_{prec}_500steps_ckpt50", "grad_q", err, floor, tol)
    jerr = abs(J - float(R["loss"])) / abs(float(R["loss"]))
    jtol = max(BAR[prec], 10 * float(R["loss_floor"])) if prec == "fp64" else BAR[prec]
    record(f"rb2d_256x128_adjoint_{prec}_500steps_ckpt50", "loss", jerr, float(R["loss_floor"]), jtol)
    assert err < tol and jerr < jtol, (err, tol, jerr, jtol)
