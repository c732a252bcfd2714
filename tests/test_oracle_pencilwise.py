"""Pin for oracle.pencilwise: the pencil-by-pencil Runge-Kutta IMEX step
equals the plain oracle step bit for bit (the same operations per pencil in
the same order), in 2D and 3D, for RK222 and RK443, with chunks that split
the pencils unevenly."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import rb, rb3d
from oracle import timesteppers as ts
from oracle.pencilwise import RungeKuttaIMEXPencilwise


@pytest.mark.parametrize("tableau", ["RK222", "RK443"])
def test_pencilwise_equals_plain_step_2d(tableau):
    sysr = rb.RB2D(32, 16, 1e6)
    X = sysr.initial_state(si.rb_noise(3, 16, 32) * 30.0)
    plain = ts.RungeKuttaIMEX(sysr, getattr(ts, tableau))
    pw = RungeKuttaIMEXPencilwise(sysr, getattr(ts, tableau), chunk=5)
    Xa, Xb = X, X
    for _ in range(2):
        Xa = plain.step(Xa, 2e-3)
        Xb = pw.step(Xb, 2e-3)
    assert np.array_equal(Xa, Xb)


def test_pencilwise_equals_plain_step_3d():
    sysr = rb3d.RB3D(8, 8, 8, 1e6)
    X = sysr.initial_state(si.rb_noise3(4, 8, 8, 8) * 30.0)
    Xa = ts.RungeKuttaIMEX(sysr).step(X, 2e-3)
    Xb = RungeKuttaIMEXPencilwise(sysr, chunk=7).step(X, 2e-3)
    assert np.array_equal(Xa, Xb)


def test_pencilwise_in_a_process_pool_equals_plain_step():
    """With a spawn pool and the problem rebuilt in the workers."""
    import functools
    import multiprocessing as mp
    from oracle.pencilwise import problem_only
    sysr = rb3d.RB3D(8, 8, 8, 1e6)
    X = sysr.initial_state(si.rb_noise3(5, 8, 8, 8) * 30.0)
    Xa = ts.RungeKuttaIMEX(sysr).step(X, 2e-3)
    factory = functools.partial(problem_only, rb3d.rb3d_problem, 8, 1e6, 1.0)
    with mp.get_context("spawn").Pool(2) as pool:
        Xb = RungeKuttaIMEXPencilwise(sysr, map_fn=pool.map, chunk=9, problem_factory=factory).step(X, 2e-3)
    assert np.array_equal(Xa, Xb)
