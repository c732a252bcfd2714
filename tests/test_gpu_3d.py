"""GPU parity of the 3D path (Fourier x, Fourier y, Chebyshev z) against the
FP64 oracle (oracle.rb3d).

* transforms at scale 1, 3/2 and 2 (order z, y, x backward; x, y, z forward);
* the seeded initial state and the dealiased advective right-hand side;
* RK222 and SBDF2 steps on a small box, FP64 (1e-12 per field, or 10x the
  oracle's own floor: SuperLU in natural order vs dense LAPACK) and mixed
  (1e-5);
* at the benchmarked size (256 x 256 x 128, one step, mixed precision):
  properties that hold at any size -- boundary rows, the divergence
  constraint and the first-order definitions -- and grid values of the
  backward transform at sampled points against the oracle's direct sums.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import bases as ob
from oracle import rb3d as orb3
from oracle import timesteppers as ots
from paper_1905_10388_gb300.solver import Context, RB3DSolver
from gpu_util import record, rel_err

pytestmark = pytest.mark.gpu
V3 = orb3.RB3D_VARIABLES


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _hermitian(c, Ny, K):
    """Coefficients of a real field: the k_x = 0 column Hermitian in k_y, the
    Nyquist y slot zero (what the forward transform of real data gives)."""
    c = c.reshape(c.shape[0], Ny, K, -1).copy()
    iy = np.arange(Ny)
    c[:, :, 0] = 0.5 * (c[:, :, 0] + np.conj(c[:, (-iy) % Ny, 0]))
    c[:, Ny // 2] = 0.0
    return c.reshape(c.shape[0], Ny * K, -1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,scale", [((16, 8, 16), (3, 2)), ((24, 16, 12), (1, 1)), ((32, 12, 8), (2, 1))])
def test_transforms_match_oracle(ctx, prec, shape, scale):
    Nx, Ny, Nz = shape
    s = RB3DSolver(ctx, Nx, Ny, Nz, 1e6, precision=prec, dealias=scale)
    sysr = orb3.RB3D(Nx, Ny, Nz, 1e6)
    rng = np.random.default_rng(Nx + Ny + Nz)
    c = rng.standard_normal((3, s.P, Nz)) + 1j * rng.standard_normal((3, s.P, Nz))
    c = _hermitian(c, Ny, Nx // 2)
    g_sz = [n * scale[0] // scale[1] for n in (Nx, Ny, Nz)]
    g = s.transform(c, -1, scale)
    ref = np.stack([sysr.to_grid(c[f], *g_sz) for f in range(3)])
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert rel_err(g, ref) < tol
    back = s.transform(ref, +1, scale)
    refc = np.stack([sysr.to_coeff(ref[f]) for f in range(3)])
    assert rel_err(back, refc) < tol
    assert np.abs(back[:, 0, :].imag).max() == 0.0


def test_initial_state_and_rhs_match_oracle(ctx):
    Nx, Ny, Nz = 16, 8, 16
    xi = si.rb_noise3(3, Nz, Ny, Nx)
    sysr = orb3.RB3D(Nx, Ny, Nz, 1e6)
    X = sysr.initial_state(xi)
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-6)):
        s = RB3DSolver(ctx, Nx, Ny, Nz, 1e6, precision=prec)
        s.factor(1e-3)
        s.set_initial_state(xi)
        got = s.get_state()
        assert rel_err(got[0], X[0]) < 1e-14
        assert rel_err(got[5], X[5]) < 1e-12
        # give the velocities content, then compare the advective terms
        rng = np.random.default_rng(1)
        Y = X.copy()
        for v in ("u", "v", "w", "uz", "vz", "wz"):
            Y[sysr.var[v]] = 1e-2 * _hermitian(rng.standard_normal((1, s.P, Nz))
                                               + 1j * rng.standard_normal((1, s.P, Nz)), Ny, Nx // 2)[0]
        s.set_state(Y)
        F = s.eval_rhs()
        Fr = sysr.nonlinear(Y)
        for e in ("b", "u", "v", "w"):
            assert rel_err(F[e], Fr[e]) < tol, (prec, e)


def _oracle_steps(Nx, Ny, Nz, Ra, xi, dt, nsteps, lu, scheme):
    sysr = orb3.RB3D(Nx, Ny, Nz, Ra, lu_method=lu)
    X = sysr.initial_state(xi)
    st = ots.RungeKuttaIMEX(sysr, getattr(ots, scheme)) if scheme.startswith("RK") else ots.SBDF(sysr, 2)
    for _ in range(nsteps):
        X = st.step(X, dt)
    return X


@pytest.mark.parametrize("kernel", ["window", "lanes"])
@pytest.mark.parametrize("scheme,prec", [("RK222", "fp64"), ("RK222", "mixed"), ("SBDF2", "fp64"), ("RK443", "fp64")])
def test_steps_match_oracle(ctx, scheme, prec, kernel):
    """Both substitution kernels against the oracle: the lane kernel is the
    one the library picks for the full-size 3D workload (32768 pencils)."""
    Nx, Ny, Nz, Ra, dt, nsteps = 16, 16, 16, 1e6, 2e-3, 5
    xi = si.rb_noise3(11, Nz, Ny, Nx) * 30.0
    s = RB3DSolver(ctx, Nx, Ny, Nz, Ra, scheme=scheme, precision=prec)
    s.set_solve_kernel(kernel)
    s.factor(dt)
    s.set_initial_state(xi)
    s.step(nsteps)
    s.sync()
    got = s.get_state()
    ref = _oracle_steps(Nx, Ny, Nz, Ra, xi, dt, nsteps, "auto", scheme)
    alt = _oracle_steps(Nx, Ny, Nz, Ra, xi, dt, nsteps, "natural", scheme)
    bar = 1e-12 if prec == "fp64" else 1e-5
    for i, v in enumerate(V3):
        floor = rel_err(alt[i], ref[i])
        err = rel_err(got[i], ref[i])
        record(f"rb3d_16x16x16_{scheme.lower()}_{prec}_{kernel}_5steps", v, err, floor, max(bar, 10 * floor))
        assert err < max(bar, 10 * floor), (v, err, floor)


def _coef_value(c, s, x, y, z):
    """Direct sum of a real field's expansion at one point (oracle bases)."""
    K, Ny, Nz = s.Nx // 2, s.Ny, s.Nz
    T = np.cos(np.arange(Nz) * np.arccos(2 * z - 1))
    kx = ob.fourier_wavenumbers(s.Nx, s.Lx)
    ky = ob.fourier_c_wavenumbers(Ny, s.Ly)
    c3 = c.reshape(Ny, K, Nz) @ T                                   # [iy, ix]
    ph = np.exp(1j * (ky[:, None] * y + kx[None, :] * x))
    w = np.where(np.arange(K) == 0, 1.0, 2.0)[None, :]
    return float(np.real(np.sum(w * c3 * ph)))


def test_full_size_one_step_properties(ctx):
    w = si.WORKLOADS["rb3d_256x256x128_rk222"]
    s = RB3DSolver(ctx, w.n_x, w.n_y, w.n_z, w.Ra, w.Pr, w.L_x, w.L_y, scheme="RK222", precision="mixed")
    s.factor(w.dt)
    s.set_initial_state(si.rb_noise3(w.seed, w.n_z, w.n_y, w.n_x))
    s.step(1)
    s.sync()
    X = s.get_state()
    var = {v: i for i, v in enumerate(V3)}
    N = w.n_z
    left, right = (-1.0) ** np.arange(N), np.ones(N)
    # boundary rows: b(0) = 1 (mean pencil), b(1) = 0, u = v = w = 0 at both walls
    bl = X[var["b"]] @ left
    assert abs(bl[0] - 1.0) < 1e-12 and np.abs(bl[1:]).max() < 1e-12
    assert np.abs(X[var["b"]] @ right).max() < 1e-12
    for f in ("u", "v"):
        assert np.abs(X[var[f]] @ left).max() < 1e-12 and np.abs(X[var[f]] @ right).max() < 1e-12
    assert np.abs(X[var["w"]] @ left).max() < 1e-12 and np.abs((X[var["w"]] @ right)[1:]).max() < 1e-12
    # divergence i k_x u + i k_y v + wz = 0, mode by mode
    kx = np.tile(ob.fourier_wavenumbers(w.n_x, w.L_x), w.n_y)[:, None]
    ky = np.repeat(ob.fourier_c_wavenumbers(w.n_y, w.L_y), w.n_x // 2)[:, None]
    div = 1j * kx * X[var["u"]] + 1j * ky * X[var["v"]] + X[var["wz"]]
    assert np.abs(div).max() < 1e-10 * max(1.0, np.abs(X[var["wz"]]).max())
    # first-order definition dz b - bz = tau U_{N-1}: its T-to-U conversion
    # vanishes in every mode but the last
    r = ob.chebyshev_derivative(X[var["b"]], 0.0, 1.0, axis=1) - X[var["bz"]]
    u = r @ ob.cheb_P_L(N).T
    assert np.abs(u[:, : N - 1]).max() < 1e-10 * np.abs(X[var["bz"]]).max()
    # backward transform at sampled points against direct sums
    g = s.get_field("b", "g")
    zs = ob.chebyshev_grid(N)
    rng = np.random.default_rng(0)
    for _ in range(6):
        iz, iy, ix = rng.integers(N), rng.integers(w.n_y), rng.integers(w.n_x)
        ref = _coef_value(X[var["b"]], s, w.L_x * ix / w.n_x, w.L_y * iy / w.n_y, zs[iz])
        assert abs(g[iz, iy, ix] - ref) < 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("case", ["3d-RK222", "3d-SBDF2", "2d-RK222", "2d-SBDF2-mixed", "3d-RK443"])
def test_lane_substitution_equals_window(ctx, case):
    """The lane-per-pencil substitution (one lane per pencil and real or
    imaginary part) performs the window kernel's FMAs in the same order, so
    SBDF2 states after several steps agree bit for bit.  For the RK schemes
    the lane path takes L~X~ of every stage but the last from that stage's
    right-hand side, (B~ - M~X~) / (H_ii dt), instead of a matvec: equal to
    rounding, which the division by H_ii dt amplifies (RK222: one such stage
    per step, 1e-12; RK443: three, 1e-11, the size of the elimination-order
    floor of the z-derivative fields at N_z = 16)."""
    from paper_1905_10388_gb300.solver import RBSolver
    dim, scheme = case.split("-")[:2]
    prec = "mixed" if case.endswith("mixed") else "fp64"
    out = []
    for kind in ("window", "lanes"):
        if dim == "3d":
            s = RB3DSolver(ctx, 16, 16, 16, 1e6, scheme=scheme, precision=prec)
            s.set_solve_kernel(kind)
            s.factor(2e-3)
            s.set_initial_state(si.rb_noise3(11, 16, 16, 16) * 30.0)
        else:
            s = RBSolver(ctx, 64, 32, 1e6, scheme=scheme, precision=prec)
            s.set_solve_kernel(kind)
            s.factor(1e-3)
            s.set_initial_state(si.rb_noise(5, 32, 64) * 30.0)
        s.step(4)
        s.sync()
        out.append(s.get_state())
        # work the kernel reports: every band entry (window) or the listed ones
        n, kl, ku = s.band()
        fma, nbytes = s.solve_work()
        if kind == "window":
            assert fma == 2 * kl + ku and nbytes == n * (2 * kl + ku + 1) * 8 + n
        else:
            assert kl < fma <= 2 * kl + ku and n * (kl + 1) * 8 < nbytes <= n * (2 * kl + ku + 1) * 8 + n
    assert np.isfinite(out[0]).all()
    if scheme == "SBDF2":
        assert np.array_equal(out[0], out[1])
    else:
        for i in range(out[0].shape[0]):
            assert rel_err(out[1][i], out[0][i]) < (1e-11 if scheme == "RK443" else 1e-12), i
