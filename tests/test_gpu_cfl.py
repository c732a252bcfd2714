"""GPU parity of the CFL control (Sec. "Timestep determination") against the
oracle (oracle.cfl).

* sp_cfl_frequency of seeded RB states, 2D and 3D, FP64 (1e-12 relative) and
  mixed (1e-6: the velocities go to the grid in FP32);
* sp_cfl_dt against the oracle rule on random inputs (the same FP64
  operations: equal);
* a CFL-driven RK222 run (the step chosen before every step, refactoring
  only when it changes): the same sequence of steps and final state as the
  oracle driven by its own controller.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import ctypes

import seeded_inputs as si
from oracle import cfl as ocfl
from oracle import rb as orb
from oracle import rb3d as orb3
from oracle import timesteppers as ots
from paper_1905_10388_gb300 import _lib as L
from paper_1905_10388_gb300.solver import CFL, Context, RB3DSolver, RBSolver
from gpu_util import field_errors

pytestmark = pytest.mark.gpu
VEL2 = (("u", "x"), ("w", "z"))
VEL3 = (("u", "x"), ("v", "y"), ("w", "z"))


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _random_state(S, P, Nz, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((S, P, Nz)) + 1j * rng.standard_normal((S, P, Nz))
    X[:, 0] = X[:, 0].real
    return X * 0.1


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_frequency_2d(ctx, prec, tol):
    Nx, Nz = 64, 32
    s = RBSolver(ctx, Nx, Nz, 1e6, precision=prec)
    s.factor(1e-3)
    sysr = orb.RB2D(Nx, Nz, 1e6)
    X = _random_state(s.S, s.P, Nz, 3)
    s.set_state(X)
    got = s.cfl_frequency(VEL2)
    ref = ocfl.frequency(sysr, X, VEL2)
    assert abs(got - ref) < tol * ref


def test_frequency_3d(ctx):
    Nx, Ny, Nz = 16, 8, 16
    s = RB3DSolver(ctx, Nx, Ny, Nz, 1e6)
    s.factor(1e-3)
    sysr = orb3.RB3D(Nx, Ny, Nz, 1e6)
    X = sysr.initial_state(si.rb_noise3(4, Nz, Ny, Nx))
    rng = np.random.default_rng(2)
    for v in ("u", "v", "w"):
        c = 0.05 * (rng.standard_normal((s.P, Nz)) + 1j * rng.standard_normal((s.P, Nz)))
        c = c.reshape(Ny, Nx // 2, Nz)
        iy = np.arange(Ny)
        c[:, 0] = 0.5 * (c[:, 0] + np.conj(c[(-iy) % Ny, 0]))   # real field: Hermitian k_x = 0 column
        c[Ny // 2] = 0.0
        X[sysr.var[v]] = c.reshape(s.P, Nz)
    s.set_state(X)
    got = s.cfl_frequency(VEL3)
    ref = ocfl.frequency(sysr, X, VEL3)
    assert abs(got - ref) < 1e-12 * ref


def test_dt_rule_matches_oracle():
    rng = np.random.default_rng(0)
    lib = L.lib()
    for _ in range(200):
        freq = float(10 ** rng.uniform(-2, 3)) if rng.random() > 0.05 else 0.0
        prev = float(10 ** rng.uniform(-4, 0)) if rng.random() > 0.1 else 0.0
        prm = (float(rng.uniform(0.1, 0.9)), float(10 ** rng.uniform(-6, -3)), float(10 ** rng.uniform(-2, 0)),
               float(rng.uniform(0.3, 0.9)), float(rng.uniform(1.1, 3.0)), float(rng.uniform(0.0, 0.3)))
        out = ctypes.c_double()
        assert lib.sp_cfl_dt(freq, prev, *prm, ctypes.byref(out)) == 0
        assert out.value == ocfl.cfl_dt(freq, prev, *prm)
    out = ctypes.c_double()
    assert lib.sp_cfl_dt(1.0, 0.1, 0.5, 1.0, 0.5, 0.5, 2.0, 0.0, ctypes.byref(out)) == L.SP_ERR_ARG


def test_cfl_driven_run_matches_oracle(ctx):
    Nx, Nz, Ra, nsteps = 32, 32, 1e5, 12
    xi = si.rb_noise(9, Nz, Nx)
    prm = dict(safety=0.3, min_dt=1e-5, max_dt=5e-3, min_change=0.5, max_change=1.5, threshold=0.05)
    s = RBSolver(ctx, Nx, Nz, Ra, scheme="RK222")
    s.factor(1e-3)
    s.set_initial_state(xi * 300.0)
    X0 = s.get_state()
    # give the flow a velocity so that the steps change
    sysr = orb.RB2D(Nx, Nz, Ra)
    rng = np.random.default_rng(1)
    for v in ("u", "w"):
        c = 0.3 * (rng.standard_normal((s.P, Nz)) + 1j * rng.standard_normal((s.P, Nz)))
        c[0] = c[0].real
        c[:, 8:] = 0.0
        X0[sysr.var[v]] = c
    s.set_state(X0)
    ctl = CFL(s, VEL2, initial_dt=1e-3, **prm)
    ctl.step(nsteps)
    s.sync()
    # the oracle driven by its own controller from the same state
    st = ots.RungeKuttaIMEX(sysr)
    X, dt, hist = X0.copy(), 1e-3, []
    for _ in range(nsteps):
        dt = ocfl.cfl_dt(ocfl.frequency(sysr, X, VEL2), dt, prm["safety"], prm["min_dt"], prm["max_dt"],
                         prm["min_change"], prm["max_change"], prm["threshold"])
        hist.append(dt)
        X = st.step(X, dt)
    assert len(set(hist)) > 2                      # the step did change
    assert np.allclose(ctl.history, hist, rtol=1e-12, atol=0)
    # a factorization exactly when the step changes
    changes = sum(1 for i in range(nsteps) if hist[i] != (hist[i - 1] if i else 1e-3))
    assert ctl.factorizations == changes
    errs = field_errors(s.get_state(), X, orb.RB_VARIABLES)
    assert max(errs.values()) < 1e-10, errs
