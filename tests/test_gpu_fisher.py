"""GPU parity of the Fisher-KPP workload (the overview example of Sec.
"Codebase structure") against the FP64 oracle (oracle.fisher).

* the example at its printed size, 128 x 64, RK222 and RK443, FP64 (1e-12 per
  field, or 10x the oracle's own floor: SuperLU in natural order vs dense
  LAPACK) and mixed (1e-5);
* the dealiased right-hand side -R u^2 of a seeded state;
* the wide channel 2048 x 1024 (the benchmarked size): three steps, mixed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import fisher as ofk
from oracle import timesteppers as ots
from paper_1905_10388_gb300.solver import Context, FisherKPPSolver
from gpu_util import rel_err

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _oracle(w, u0, scheme, nsteps, lu):
    sysr = ofk.FisherKPP(w.n_x, w.n_z, w.D, w.R, w.L_x, lu_method=lu)
    X = sysr.initial_state(u0)
    st = ots.RungeKuttaIMEX(sysr, getattr(ots, scheme))
    for _ in range(nsteps):
        X = st.step(X, w.dt)
    return X


def _gpu(ctx, w, u0, scheme, nsteps, prec):
    s = FisherKPPSolver(ctx, w.n_x, w.n_z, w.D, w.R, w.L_x, scheme=scheme, precision=prec)
    s.factor(w.dt)
    s.set_initial_state(u0)
    s.step(nsteps)
    s.sync()
    return s.get_state()


@pytest.mark.parametrize("scheme,prec", [("RK222", "fp64"), ("RK222", "mixed"), ("RK443", "fp64")])
def test_fisher_128x64_matches_oracle(ctx, scheme, prec):
    w = si.WORKLOADS["fisher_128x64_rk222"]
    nsteps = 40
    u0 = si.fisher_noise(w.seed, w.n_z, w.n_x)
    got = _gpu(ctx, w, u0, scheme, nsteps, prec)
    ref = _oracle(w, u0, scheme, nsteps, "auto")
    alt = _oracle(w, u0, scheme, nsteps, "natural")
    for i, v in enumerate(ofk.FISHER_VARIABLES):
        floor = rel_err(alt[i], ref[i])
        err = rel_err(got[i], ref[i])
        assert err < max(TOL[prec], 10 * floor), (v, err, floor)


def test_fisher_rhs_matches_oracle(ctx):
    w = si.WORKLOADS["fisher_128x64_rk222"]
    u0 = si.fisher_noise(w.seed + 1, w.n_z, w.n_x)
    sysr = ofk.FisherKPP(w.n_x, w.n_z, w.D, w.R, w.L_x)
    X = sysr.initial_state(u0)
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-6)):
        s = FisherKPPSolver(ctx, w.n_x, w.n_z, w.D, w.R, w.L_x, precision=prec)
        s.factor(w.dt)
        s.set_state(X)
        F = s.eval_rhs()
        assert rel_err(F["u"], sysr.nonlinear(X)["u"]) < tol, prec


def test_fisher_2048x1024_three_steps(ctx):
    w = si.WORKLOADS["fisher_2048x1024_rk222"]
    nsteps = 3
    u0 = si.fisher_noise(w.seed, w.n_z, w.n_x)
    got = _gpu(ctx, w, u0, "RK222", nsteps, "mixed")
    ref = _oracle(w, u0, "RK222", nsteps, "auto")
    for i, v in enumerate(ofk.FISHER_VARIABLES):
        assert rel_err(got[i], ref[i]) < TOL["mixed"], v
