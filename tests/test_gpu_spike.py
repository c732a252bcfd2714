"""GPU parity of the partitioned substitution (row blocks substituted in
parallel, inflows by a recurrence over blocks; Sec. "Matrix solvers").

* against the FP64 oracle at sizes the oracle finishes quickly, for several
  block counts and schemes, with the per-field bar of the other FP64 parity
  tests (1e-12 or 10 x the oracle variants' floor) and mixed 1e-5;
* against the whole-row-order window kernel on the benchmarked 512 x 256
  SBDF2 problem (the same arithmetic per row, the inflows summed in another
  order: equal to rounding);
* every block count of that problem gives the same state to rounding;
* the library picks it automatically for that problem.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import rb as orb
from oracle import timesteppers as ots
from paper_1905_10388_gb300.solver import Context, RBSolver
from gpu_util import check_fields, oracle_floor, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _solver(ctx, nx, nz, ra, scheme, prec, kind, nblk=0):
    s = RBSolver(ctx, nx, nz, ra, scheme=scheme, precision=prec)
    s.set_solve_kernel(kind)
    if nblk:
        s.set_spike_blocks(nblk)
    return s


@pytest.mark.parametrize("scheme,prec,nblk", [("RK222", "fp64", 2), ("RK222", "fp64", 7), ("RK222", "mixed", 14),
                                              ("SBDF2", "fp64", 14), ("RK443", "fp64", 7)])
def test_spike_matches_oracle(ctx, scheme, prec, nblk):
    nx, nz, ra, dt, nsteps = 64, 64, 1e6, 1e-3, 6
    xi = si.rb_noise(21, nz, nx) * 30.0
    s = _solver(ctx, nx, nz, ra, scheme, prec, "spike", nblk)
    s.factor(dt)
    assert s.spike_blocks() == nblk
    s.set_initial_state(xi)
    s.step(nsteps)
    ctx.sync_status()

    def stepper(sysr):
        st = ots.RungeKuttaIMEX(sysr, getattr(ots, scheme)) if scheme.startswith("RK") else ots.SBDF(sysr, 2)
        st.dt = dt
        return st
    ref, floor = oracle_floor(lambda m, lu: orb.RB2D(nx, nz, ra, cheb_method=m, lu_method=lu),
                              lambda sysr: sysr.initial_state(xi), stepper, nsteps)
    check_fields(s.get_state(), ref, floor, 1e-12 if prec == "fp64" else 1e-5,
                 label=f"spike_64x64_{scheme.lower()}_{prec}_nblk{nblk}_6steps")


def test_spike_rejects_blocks_that_split_a_chunk(ctx):
    """64 x 64: 448 rows = 14 chunks of 32; 4 blocks would split a chunk."""
    from paper_1905_10388_gb300 import _lib as L
    s = RBSolver(ctx, 64, 64, 1e6)
    with pytest.raises(L.SpectauError):
        s.set_spike_blocks(4)


def test_spike_equals_window_at_512x256(ctx):
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    out = {}
    for kind in ("window", "spike"):
        s = _solver(ctx, w.n_x, w.n_z, w.Ra, "SBDF2", "fp64", kind)
        s.factor(w.dt)
        s.set_initial_state(xi)
        s.step(20, graph=True)
        ctx.sync_status()
        out[kind] = s.get_state()
    for i, v in enumerate(orb.RB_VARIABLES):
        assert rel_err(out["spike"][i], out["window"][i]) < 1e-11, v


def test_spike_block_counts_agree_and_auto_choice(ctx):
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    auto = RBSolver(ctx, w.n_x, w.n_z, w.Ra, scheme="SBDF2")
    auto.factor(w.dt)
    assert auto.spike_blocks() > 1          # 256 pencils of 1792 rows: partitioned by default
    states = []
    for nblk in (2, 4, 7, 8, 14, 28, 56):
        s = _solver(ctx, w.n_x, w.n_z, w.Ra, "SBDF2", "fp64", "spike", nblk)
        s.factor(w.dt)
        s.set_initial_state(xi)
        s.step(5)
        ctx.sync_status()
        states.append(s.get_state())
    for X in states[1:]:
        for i, v in enumerate(orb.RB_VARIABLES):
            assert rel_err(X[i], states[0][i]) < 1e-11, v


def test_spike_graph_equals_eager(ctx):
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    res = []
    for graph in (False, True):
        s = _solver(ctx, w.n_x, w.n_z, w.Ra, "SBDF2", "mixed", "spike")
        s.factor(w.dt)
        s.set_initial_state(xi)
        s.step(7, graph=graph)
        ctx.sync_status()
        res.append(s.get_state())
    assert np.array_equal(res[0], res[1])
