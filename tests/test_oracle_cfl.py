"""Pins for oracle.cfl (Sec. "Timestep determination").

* a uniform x-flow U has frequency U N_gx / L_x everywhere;
* the z spacing is numpy's gradient of the dealiased Chebyshev nodes, and a
  uniform z-flow W has frequency W / min spacing (at the walls);
* the rule: safety / frequency, the absolute and relative bounds and the
  threshold on hand-worked cases.
"""
import numpy as np

from oracle import bases
from oracle import cfl
from oracle import rb as orb


def test_uniform_x_flow():
    s = orb.RB2D(16, 12, 1e5)
    X = np.zeros((s.S, s.P, s.Nz), complex)
    X[s.var["u"], 0, 0] = 0.7                                  # u = 0.7 everywhere
    f = cfl.frequency(s, X, (("u", "x"), ("w", "z")))
    assert abs(f - 0.7 * s.Ngx / s.Lx) < 1e-13


def test_z_spacing_is_the_node_gradient_and_uniform_z_flow():
    n = 18
    assert np.allclose(cfl.z_spacing(n), np.gradient(bases.chebyshev_grid(n)), rtol=0, atol=1e-15)
    s = orb.RB2D(8, 12, 1e5)
    X = np.zeros((s.S, s.P, s.Nz), complex)
    X[s.var["w"], 0, 0] = -0.3
    f = cfl.frequency(s, X, (("u", "x"), ("w", "z")))
    d = np.gradient(bases.chebyshev_grid(s.Ngz))
    assert abs(f - 0.3 / d.min()) < 1e-12 * f


def test_rule_cases():
    # safety / freq inside every bound
    assert cfl.cfl_dt(10.0, 0.04, 0.5, 0.0, 1.0, 0.5, 2.0, 0.0) == 0.05
    # absolute cap, then the relative cap against the previous step
    assert cfl.cfl_dt(0.1, 0.04, 0.5, 0.0, 1.0, 0.5, 2.0, 0.0) == 0.08
    assert cfl.cfl_dt(0.1, 0.0, 0.5, 0.0, 1.0, 0.5, 2.0, 0.0) == 1.0
    # relative floor
    assert cfl.cfl_dt(1000.0, 0.04, 0.5, 0.0, 1.0, 0.5, 2.0, 0.0) == 0.02
    # below the threshold the previous step is kept; above it, not
    assert cfl.cfl_dt(10.0, 0.048, 0.5, 0.0, 1.0, 0.5, 2.0, 0.1) == 0.048
    assert cfl.cfl_dt(10.0, 0.04, 0.5, 0.0, 1.0, 0.5, 2.0, 0.1) == 0.05
    # no flow: max_dt
    assert cfl.cfl_dt(0.0, 0.0, 0.5, 0.0, 0.3, 0.5, 2.0, 0.0) == 0.3
