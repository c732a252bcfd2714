"""The Chebyshev backward transform on the tensor cores (tcgen05.mma
kind::tf32 with a three-product TF32 split, operands staged by TMA) against
the FP64 oracle, in the mixed form (bar 1e-5 per field):

* the dealiased advective right-hand side (every grid field: values and the
  i k_x, i k_y multiples taken in the epilogue) in 2D and 3D;
* RK222 steps in 2D and 3D against the oracle;
* the tensor-core and FFT paths agree far below the bar;
* sizes and precisions the kernel does not take are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import rb as orb
from oracle import rb3d as orb3
from oracle import timesteppers as ots
from paper_1905_10388_gb300 import _lib
from paper_1905_10388_gb300.solver import Context, RB3DSolver, RBSolver
from gpu_util import check_fields, oracle_floor, record, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _rhs_state_2d(nx, nz):
    sysr = orb.RB2D(nx, nz, 1e6)
    X = sysr.initial_state(si.rb_noise(5, nz, nx))
    rng = np.random.default_rng(3)
    for v in ("u", "w", "uz", "wz"):
        c = 1e-2 * (rng.standard_normal((sysr.P, nz)) + 1j * rng.standard_normal((sysr.P, nz)))
        c[0] = c[0].real
        X[sysr.var[v]] = c
    return sysr, X


@pytest.mark.parametrize("nx,nz", [(64, 64), (32, 32), (128, 128)])
def test_rhs_2d_mma_matches_oracle_and_fft(ctx, nx, nz):
    sysr, X = _rhs_state_2d(nx, nz)
    ref = sysr.nonlinear(X)
    out = {}
    for kind in ("mma", "fft"):
        s = RBSolver(ctx, nx, nz, 1e6, precision="mixed")
        s.set_z_transform(kind)
        s.factor(1e-3)
        assert s.z_transform() == kind
        s.set_state(X)
        out[kind] = s.eval_rhs()
    for e in ("b", "u", "w"):
        err = rel_err(out["mma"][e], ref[e])
        record(f"chebmma_rhs_2d_{nx}x{nz}", e, err, None, 1e-5)
        assert err < 1e-5, (e, err)
        assert rel_err(out["mma"][e], out["fft"][e]) < 5e-6


def test_rk222_2d_mma_matches_oracle(ctx):
    nx, nz, ra, dt, nsteps = 64, 64, 1e6, 1e-3, 6
    xi = si.rb_noise(21, nz, nx) * 30.0
    s = RBSolver(ctx, nx, nz, ra, scheme="RK222", precision="mixed")
    s.set_z_transform("mma")
    s.factor(dt)
    s.set_initial_state(xi)
    s.step(nsteps)
    ctx.sync_status()

    def stepper(sysr):
        st = ots.RungeKuttaIMEX(sysr)
        st.dt = dt
        return st
    ref, floor = oracle_floor(lambda m, lu: orb.RB2D(nx, nz, ra, cheb_method=m, lu_method=lu),
                              lambda sysr: sysr.initial_state(xi), stepper, nsteps)
    check_fields(s.get_state(), ref, floor, 1e-5, label="chebmma_rk222_2d_64x64_mixed_6steps")


def test_3d_auto_uses_mma_and_matches_oracle(ctx):
    Nx, Ny, Nz, Ra, dt, nsteps = 16, 16, 32, 1e6, 2e-3, 4
    xi = si.rb_noise3(11, Nz, Ny, Nx) * 30.0
    s = RB3DSolver(ctx, Nx, Ny, Nz, Ra, scheme="RK222", precision="mixed")
    s.factor(dt)
    assert s.z_transform() == "mma"
    s.set_initial_state(xi)
    s.step(nsteps)
    ctx.sync_status()
    sysr = orb3.RB3D(Nx, Ny, Nz, Ra)
    X = sysr.initial_state(xi)
    st = ots.RungeKuttaIMEX(sysr)
    for _ in range(nsteps):
        X = st.step(X, dt)
    got = s.get_state()
    for i, v in enumerate(orb3.RB3D_VARIABLES):
        err = rel_err(got[i], X[i])
        record("chebmma_rk222_3d_16x16x32_mixed_4steps", v, err, None, 1e-5)
        assert err < 1e-5, (v, err)


def test_mma_refuses_what_it_does_not_take(ctx):
    s = RBSolver(ctx, 64, 64, 1e6, precision="fp64")
    with pytest.raises(_lib.SpectauError):
        s.set_z_transform("mma")
    s = RBSolver(ctx, 64, 16, 1e6, precision="mixed")     # N_z = 16: not a multiple of 32
    with pytest.raises(_lib.SpectauError):
        s.set_z_transform("mma")
    s = RBSolver(ctx, 64, 256, 1e6, precision="mixed")    # N_gz = 384: more than one MMA's N (256)
    with pytest.raises(_lib.SpectauError):
        s.set_z_transform("mma")
