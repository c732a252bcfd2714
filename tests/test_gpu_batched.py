"""Batched stepping of uneven problems (one launch per kernel type per stage).

The batched kernels run the same device code per item as the single-problem
kernels, so a batch must reproduce each problem stepped alone bit for bit;
a sample of instances is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import rb as orb
from oracle import timesteppers as ots
from paper_1905_10388_gb300.solver import (Context, RBSolver, batch_persistent, batch_tile, set_batch_persistent,
                                           step_batched)
from gpu_util import check_fields, oracle_floor

pytestmark = pytest.mark.gpu

SHAPES = [(32, 16, 3e5), (64, 32, 1e6), (128, 64, 2e7), (64, 16, 1e5), (32, 64, 5e7), (128, 32, 1e6)]


def _make(ctx, scheme, prec, seed0=1000):
    out = []
    for i, (nx, nz, ra) in enumerate(SHAPES):
        s = RBSolver(ctx, nx, nz, ra, scheme=scheme, precision=prec)
        s.factor(1e-3 * 32.0 / nz)
        s.set_initial_state(si.rb_noise(seed0 + i, nz, nx))
        out.append(s)
    return out


@pytest.mark.parametrize("scheme,prec,graph", [("RK222", "fp64", False), ("RK222", "mixed", True),
                                               ("SBDF2", "fp64", True), ("RK443", "mixed", True)])
def test_batch_equals_individual_steps(scheme, prec, graph):
    ctx = Context(0)
    solo = _make(ctx, scheme, prec)
    for s in solo:
        s.step(9)
    batch = _make(ctx, scheme, prec)
    step_batched(batch, 9, graph=graph)
    ctx.sync_status()
    assert batch_tile(batch) in (4, 8, 16)
    for a, b in zip(solo, batch):
        assert np.array_equal(a.get_state(), b.get_state())
    ctx.close()


@pytest.mark.parametrize("scheme", ["SBDF3", "SBDF4", "CNAB2"])
def test_batch_multistep_phases_equal_individual_steps(scheme):
    """Multistep schemes rotate history rings of depth D (SBDF3: 3, SBDF4: 4,
    CNAB2: 2): the batch keeps one set of launch tables per phase and must
    still equal the problems stepped alone, bit for bit."""
    ctx = Context(0)
    solo = _make(ctx, scheme, "fp64")
    for s in solo:
        s.step(11)
    batch = _make(ctx, scheme, "fp64")
    step_batched(batch, 11, graph=True)
    ctx.sync_status()
    for a, b in zip(solo, batch):
        assert np.array_equal(a.get_state(), b.get_state())
    ctx.close()


def test_batch_sample_against_oracle():
    ctx = Context(0)
    batch = _make(ctx, "RK222", "fp64")
    step_batched(batch, 4, graph=True)
    ctx.sync_status()
    for i in (0, 2, 4):
        nx, nz, ra = SHAPES[i]
        dt = 1e-3 * 32.0 / nz

        class _RK(ots.RungeKuttaIMEX):
            pass

        def stepper(sysr):
            st = _RK(sysr)
            st.dt = dt
            return st
        ref, floor = oracle_floor(lambda m, lu: orb.RB2D(nx, nz, ra, cheb_method=m, lu_method=lu),
                                  lambda sysr: sysr.initial_state(si.rb_noise(1000 + i, nz, nx)), stepper, 4)
        check_fields(batch[i].get_state(), ref, floor, 1e-12, label=f"batch_sample_{nx}x{nz}_rk222_fp64_4steps")
    ctx.close()


@pytest.mark.parametrize("scheme", ["RK222", "SBDF2"])
def test_batch_after_refactor_equals_individual_steps(scheme):
    """A batch caches each problem's factor and step coefficients in its
    argument tables and graphs; re-factoring at a new dt must drop that cache,
    so batch steps after the re-factor equal individual steps bit for bit."""
    ctx = Context(0)
    solo = _make(ctx, scheme, "fp64")
    batch = _make(ctx, scheme, "fp64")
    for s in solo:
        s.step(4)
    step_batched(batch, 4, graph=True)
    for s in solo + batch:
        s.factor(0.5e-3 * 32.0 / s.Nz)
    for s in solo:
        s.step(5)
    step_batched(batch, 5, graph=True)
    ctx.sync_status()
    for a, b in zip(solo, batch):
        assert np.array_equal(a.get_state(), b.get_state())
    ctx.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_persistent_and_per_item_launches_agree(persistent):
    """Both launch shapes of the batched kernels (one CTA per work item, and
    persistent grids pulling items from device counters) compute every item
    with the same code: the states after 5 steps equal the problems stepped
    alone bit for bit."""
    ctx = Context(0)
    solo = _make(ctx, "RK222", "mixed")
    for s in solo:
        s.step(5)
    batch = _make(ctx, "RK222", "mixed")
    set_batch_persistent(batch, persistent)
    step_batched(batch, 5, graph=True)
    ctx.sync_status()
    assert batch_persistent(batch) == persistent
    for a, b in zip(solo, batch):
        assert np.array_equal(a.get_state(), b.get_state())
    ctx.close()
