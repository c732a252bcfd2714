"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds workload sizes and random draws only -- none of the
method's arithmetic -- so that both the CUDA path and the oracle can take the
identical inputs without sharing any code of the method.

Rayleigh-Benard initial state recipe (used by both sides): the buoyancy on
the scale-1 grid is b = 1 - z + A xi(z, x) z (1 - z) with A = 1e-3 and xi
i.i.d. standard normals of shape (N_z, N_x) (row = Chebyshev node in
ascending z, column = Fourier node), drawn in C order from
``numpy.random.default_rng(seed).standard_normal``.  Each side turns xi into
coefficients with its own transforms.

Fisher-KPP initial state recipe: u on the scale-1 grid is i.i.d. uniform on
[0, 1), shape (N_z, N_x), from ``numpy.random.default_rng(seed).random``
(the overview example's random initial values, seeded).
"""
from dataclasses import dataclass, field

import numpy as np

NOISE_AMPLITUDE = 1e-3


@dataclass(frozen=True)
class RBWorkload:
    name: str
    n_x: int
    n_z: int
    Ra: float
    Pr: float = 1.0
    L_x: float = 4.0
    scheme: str = "RK222"
    dt: float = 1e-3
    steps: int = 100
    seed: int = 42
    n_y: int = 1
    L_y: float = 4.0

    @property
    def dof(self):
        """Real unknowns S * N_x * N_y * N_z (S = 7 fields in 2D, 9 in 3D)."""
        s = 7 if self.n_y == 1 else 9
        return s * self.n_x * self.n_y * self.n_z

    @property
    def modes(self):
        return self.n_x * self.n_y * self.n_z


@dataclass(frozen=True)
class FisherWorkload:
    """Fisher-KPP channel: N_x Fourier modes on [0, L_x), N_z Chebyshev on [0, 1]."""
    name: str
    n_x: int
    n_z: int
    D: float = 0.1
    R: float = 1.0
    L_x: float = 2 * np.pi
    scheme: str = "RK222"
    dt: float = 0.01
    steps: int = 200
    seed: int = 42
    n_y: int = 1

    @property
    def dof(self):
        """Real unknowns S * N_x * N_z (S = 2: u, uz)."""
        return 2 * self.n_x * self.n_z

    @property
    def modes(self):
        return self.n_x * self.n_z


# The five workloads.  Small one: 2D 64x32 RK222.  Headline: 2D 512x256 SBDF2.
WORKLOADS = {
    "rb2d_64x32_rk222": RBWorkload("rb2d_64x32_rk222", 64, 32, 1e6, scheme="RK222",
                                   dt=1e-3, steps=100),
    "rb2d_512x256_sbdf2": RBWorkload("rb2d_512x256_sbdf2", 512, 256, 1e8, scheme="SBDF2",
                                     dt=1e-4, steps=1000),
    "rb3d_256x256x128_rk222": RBWorkload("rb3d_256x256x128_rk222", 256, 128, 1e7,
                                         scheme="RK222", dt=5e-4, steps=200, n_y=256),
    "rb2d_256x128_rk222_adjoint": RBWorkload("rb2d_256x128_rk222_adjoint", 256, 128, 1e6,
                                             scheme="RK222", dt=1e-3, steps=500),
    # the benchmarked 2D workload with the third-order four-stage RK443
    "rb2d_512x256_rk443": RBWorkload("rb2d_512x256_rk443", 512, 256, 1e8, scheme="RK443",
                                     dt=1e-4, steps=1000),
    # the overview example at its printed size (128 x 64, D = 0.1, R = 1,
    # RK222, dt = 0.01) and a wider channel
    "fisher_128x64_rk222": FisherWorkload("fisher_128x64_rk222", 128, 64),
    "fisher_2048x1024_rk222": FisherWorkload("fisher_2048x1024_rk222", 2048, 1024, dt=1e-3),
    # profiling slab of the 3D workload: the same 32768 pencils with 16
    # Chebyshev modes (about 2.5 GB on the device instead of about 25 GB)
    "rb3d_256x256x16_rk222": RBWorkload("rb3d_256x256x16_rk222", 256, 16, 1e7,
                                        scheme="RK222", dt=5e-4, steps=200, n_y=256),
    # profiling case of the 3D z transforms: 128 Chebyshev modes (N_gz = 192,
    # the tensor-core path's size) on 64 x 64 Fourier modes, 2048 pencils
    # (about 1.6 GB on the device)
    "rb3d_64x64x128_rk222": RBWorkload("rb3d_64x64x128_rk222", 64, 128, 1e7,
                                       scheme="RK222", dt=5e-4, steps=200, n_y=64),
}


def rb_noise(seed, n_z, n_x):
    """xi[z, x]: i.i.d. standard normals on the scale-1 grid."""
    return np.random.default_rng(seed).standard_normal((n_z, n_x))


def rb_noise3(seed, n_z, n_y, n_x):
    """xi[z, y, x]: i.i.d. standard normals on the 3D scale-1 grid."""
    return np.random.default_rng(seed).standard_normal((n_z, n_y, n_x))


def batched_workloads(count=64, seed=7):
    """Uneven batch: N_x from {64..512}, N_z from {32..256}, Ra log-uniform."""
    rng = np.random.default_rng(seed)
    nx = rng.choice([64, 128, 256, 512], size=count)
    nz = rng.choice([32, 64, 128, 256], size=count)
    ra = 10.0 ** rng.uniform(5.0, 8.0, size=count)
    out = []
    for i in range(count):
        out.append(RBWorkload(f"batch{i}", int(nx[i]), int(nz[i]), float(ra[i]),
                              scheme="RK222", dt=1e-3 * 32.0 / float(nz[i]),
                              steps=500, seed=1000 + i))
    return out


def fisher_noise(seed, n_z, n_x):
    """u[z, x]: i.i.d. uniform on [0, 1) on the scale-1 grid."""
    return np.random.default_rng(seed).random((n_z, n_x))
