"""CFL timestep control (oracle; test infrastructure): Sec. "Timestep
determination".

frequency(system, X, velocities): at every point of the dealiased grid the
velocity magnitudes divided by the local grid spacing are added; the largest
sum over the grid is returned.  Spacing: L_x / N_gx (and L_y / N_gy) on the
Fourier axes; on z the centred difference of neighbouring Chebyshev nodes,
one-sided at the two end nodes.

cfl_dt(...): the step is safety / frequency, limited to [min_dt, max_dt],
then to [min_change, max_change] times the previous step, and the previous
step is kept when the fractional change is below the threshold.

Pins: ``tests/test_oracle_cfl.py`` (a uniform flow gives U N_gx / L_x; the
z spacing is numpy's gradient of the nodes; the rule's branches on
hand-worked cases).
"""
import numpy as np

from . import bases


def z_spacing(n_g, a=0.0, b=1.0):
    z = bases.chebyshev_grid(n_g, a, b)
    d = np.empty(n_g)
    d[1:-1] = 0.5 * (z[2:] - z[:-2])
    d[0], d[-1] = z[1] - z[0], z[-1] - z[-2]
    return d


def frequency(system, X, velocities):
    """velocities: ((variable, axis), ...), axis 'x', 'y' or 'z'; the grid
    is the system's dealiased grid, g[z, x] (2D) or g[z, y, x] (3D)."""
    total = 0.0
    for var, axis in velocities:
        g = np.abs(system.to_grid(X[system.var[var]]))
        if axis == "x":
            inv = system.Ngx / system.Lx
        elif axis == "y":
            inv = system.Ngy / system.Ly
        else:
            inv = 1.0 / z_spacing(system.Ngz)
            inv = inv.reshape((-1,) + (1,) * (g.ndim - 1))
        total = total + g * inv
    return float(np.max(total))


def cfl_dt(freq, dt_prev, safety, min_dt, max_dt, min_change, max_change, threshold):
    dt = safety / freq if freq > 0 else max_dt
    dt = min(max(dt, min_dt), max_dt)
    if dt_prev > 0:
        dt = min(max(dt, min_change * dt_prev), max_change * dt_prev)
        if abs(dt - dt_prev) < threshold * dt_prev:
            dt = dt_prev
    return dt
