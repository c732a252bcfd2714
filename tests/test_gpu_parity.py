"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: the all-FP64 form must match to 1e-12 relative per field (the
target of the method's FP64 form); the mixed form (FP32 transforms and
products, FP64 pencils) to 1e-5 relative per field.  Errors are
||x_gpu - x_ref||_2 / ||x_ref||_2 over each field's coefficients (absolute
when the reference norm is below 1e-30).

Where FP64 evaluations of the same definition already differ by more than
the bar (the rounding floor: the largest deviation of oracle variants that
sum the Chebyshev transforms by scipy's DCT instead of the T_n(x_i)
quadrature and/or eliminate the pencils with SuperLU in natural order
instead of dense LAPACK), the bar for that field is 10x the floor.  This
bites only for the z-derivative fields (bz, uz), whose relative error is
set by the conditioning of the pencil solves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import seeded_inputs as si
from oracle import bases as ob
from oracle import rb as orb
from oracle import timesteppers as ots
from paper_1905_10388_gb300 import _lib
from paper_1905_10388_gb300.solver import Context, RBSolver
from gpu_util import check_fields, FLOOR_VARIANTS, field_errors, rel_err

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _oracle_run(sysr, X, scheme, dt, nsteps):
    if scheme == "RK222":
        st = ots.RungeKuttaIMEX(sysr)
    elif scheme in ("RK111", "RK443"):
        st = ots.RungeKuttaIMEX(sysr, getattr(ots, scheme))
    elif scheme.startswith("CNAB"):
        st = ots.CNAB(sysr, int(scheme[-1]))
    else:
        st = ots.SBDF(sysr, int(scheme[-1]))
    for _ in range(nsteps):
        X = st.step(X, dt)
    return X


_REF_CACHE = {}


def _reference(n_x, n_z, Ra, xi, scheme, dt, nsteps, Pr=1.0, L_x=4.0, dealias=1.5):
    """Oracle result and per-field rounding floor (largest deviation of the
    oracle variants that sum the same arithmetic in other orders)."""
    key = (n_x, n_z, Ra, xi.tobytes(), scheme, dt, nsteps, Pr, L_x, dealias)
    if key in _REF_CACHE:
        return _REF_CACHE[key]
    out = []
    for cheb, lu in (("mmt", "auto"),) + FLOOR_VARIANTS:
        sysr = orb.RB2D(n_x, n_z, Ra, Pr, L_x, dealias=dealias, cheb_method=cheb, lu_method=lu)
        out.append(_oracle_run(sysr, sysr.initial_state(xi), scheme, dt, nsteps))
    floor = dict.fromkeys(orb.RB_VARIABLES, 0.0)
    for X in out[1:]:
        for k, v in field_errors(X, out[0], orb.RB_VARIABLES).items():
            floor[k] = max(floor[k], v)
    _REF_CACHE[key] = (out[0], floor)
    return out[0], floor


def _check(got, ref, floor, bar, label=None):
    """Per field: error below max(bar, 10 x floor); every figure is recorded
    under the running test's id."""
    import os
    label = label or os.environ.get("PYTEST_CURRENT_TEST", "parity").split(" ")[0]
    check_fields(got, ref, floor, bar, label=label)


# --- transforms (Sec. "Scaled transforms & dealiasing") ----------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("Nx,Nz,scale", [(64, 32, (3, 2)), (24, 24, (1, 1)), (128, 64, (3, 2)), (48, 12, (2, 1))])
def test_transforms_match_oracle(ctx, prec, Nx, Nz, scale):
    s = RBSolver(ctx, Nx, Nz, 1e6, precision=prec, dealias=scale)
    sysr = orb.RB2D(Nx, Nz, 1e6)
    rng = np.random.default_rng(Nx + Nz)
    P = Nx // 2
    c = rng.standard_normal((3, P, Nz)) + 1j * rng.standard_normal((3, P, Nz))
    c[:, 0, :] = c[:, 0, :].real
    ngx, ngz = Nx * scale[0] // scale[1], Nz * scale[0] // scale[1]
    g = s.transform(c, -1, scale)
    ref = np.stack([sysr.to_grid(c[f], ngx, ngz) for f in range(3)])
    assert rel_err(g, ref) < (1e-13 if prec == "fp64" else 2e-6)
    back = s.transform(ref, +1, scale)
    refc = np.stack([ob.chebyshev_forward(ob.fourier_forward(ref[f], Nx, axis=1), Nz, axis=0).T for f in range(3)])
    assert rel_err(back, refc) < (1e-13 if prec == "fp64" else 2e-6)
    assert np.abs(back[:, 0, :].imag).max() == 0.0          # Im f_0 = 0 for real data


def test_grid_state_round_trip_and_dz(ctx):
    Nx, Nz = 32, 16
    s = RBSolver(ctx, Nx, Nz, 1e6)
    s.factor(1e-3)
    xi = si.rb_noise(11, Nz, Nx)
    s.set_initial_state(xi)
    sysr = orb.RB2D(Nx, Nz, 1e6)
    X = sysr.initial_state(xi)
    assert rel_err(s.get_field("b"), X[0]) < 1e-14
    assert rel_err(s.get_field("bz"), X[4]) < 1e-12   # O(N) recurrence vs dense D^TT
    z = ob.chebyshev_grid(Nz)[:, None]
    bg = 1 - z + 1e-3 * xi * z * (1 - z)
    nyq = (bg * (-1.0) ** np.arange(Nx)).mean(axis=1, keepdims=True) * (-1.0) ** np.arange(Nx)
    assert np.abs(s.get_field("b", "g") - (bg - nyq)).max() < 1e-14


# --- nonlinear RHS --------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bilinear_rhs_matches_oracle(ctx, prec):
    Nx, Nz = 64, 32
    sysr = orb.RB2D(Nx, Nz, 1e6)
    X = sysr.initial_state(si.rb_noise(5, Nz, Nx))
    rng = np.random.default_rng(3)
    for v in (2, 3, 5, 6):          # give u, w, uz, wz some content
        X[v] = 1e-2 * (rng.standard_normal(X[v].shape) + 1j * rng.standard_normal(X[v].shape))
        X[v][0] = X[v][0].real
    s = RBSolver(ctx, Nx, Nz, 1e6, precision=prec)
    s.factor(1e-3)
    s.set_state(X)
    F = s.eval_rhs()
    Fr = sysr.nonlinear(X)
    for e in ("b", "u", "w"):
        assert rel_err(F[e], Fr[e]) < (1e-13 if prec == "fp64" else 1e-6), e


# --- full steps -------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rb_64x32_rk222_100_steps(ctx, prec):
    w = si.WORKLOADS["rb2d_64x32_rk222"]
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK222", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(xi)
    s.step(w.steps)
    s.sync()
    ref, floor = _reference(w.n_x, w.n_z, w.Ra, xi, "RK222", w.dt, w.steps, w.Pr, w.L_x)
    _check(s.get_state(), ref, floor, TOL[prec])


@pytest.mark.parametrize("scheme", ["SBDF2", "SBDF1", "RK111", "RK443", "SBDF3", "SBDF4", "CNAB1", "CNAB2"])
def test_rb_small_other_schemes(ctx, scheme):
    """12 steps; CNAB 11: Crank-Nicolson leaves the pressure (an algebraic
    variable) alternating about its mean, p^{n+1} = 2 p_mean - p^n, so from
    p^0 = 0 the pressure at an even step is the cancelled remainder of an
    O(1) hydrostatic field and its relative error is no measure of anything."""
    Nx, Nz, Ra, dt = 32, 32, 1e5, 2e-3
    nsteps = 11 if scheme.startswith("CNAB") else 12
    xi = si.rb_noise(9, Nz, Nx)
    s = RBSolver(ctx, Nx, Nz, Ra, scheme=scheme)
    s.factor(dt)
    s.set_initial_state(xi)
    s.step(nsteps)
    s.sync()
    ref, floor = _reference(Nx, Nz, Ra, xi, scheme, dt, nsteps)
    _check(s.get_state(), ref, floor, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rb_512x256_sbdf2_full_size(ctx, prec):
    """The benchmarked workload at full size: a few SBDF2 steps (SBDF1 start)."""
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    nsteps = 3
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="SBDF2", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(xi)
    s.step(nsteps)
    s.sync()
    ref, floor = _reference(w.n_x, w.n_z, w.Ra, xi, "SBDF2", w.dt, nsteps, w.Pr, w.L_x)
    _check(s.get_state(), ref, floor, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rb_512x256_rk443_full_size(ctx, prec):
    """The benchmarked 2D size with the four-stage RK443: two steps (eight
    stage solves with one factor, L~X~^j of three stages carried)."""
    w = si.WORKLOADS["rb2d_512x256_rk443"]
    nsteps = 2
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK443", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(xi)
    s.step(nsteps)
    s.sync()
    ref, floor = _reference(w.n_x, w.n_z, w.Ra, xi, "RK443", w.dt, nsteps, w.Pr, w.L_x)
    _check(s.get_state(), ref, floor, TOL[prec])


def test_ragged_pencil_tiles(ctx):
    # P = 12 pencils: not a multiple of the z-kernel tile of 8
    Nx, Nz, Ra, dt = 24, 12, 1e5, 1e-3
    xi = si.rb_noise(4, Nz, Nx)
    from paper_1905_10388_gb300 import rb as prb
    from paper_1905_10388_gb300.solver import TauSolver
    s = TauSolver(ctx, prb.rb_pencil_problem(Ra), Nx, Nz, 4.0, scheme="RK222", dealias=(2, 1),
                  bilinear=prb.BILINEAR_TERMS)
    s.state_order = prb.VARIABLES
    s.factor(dt)
    z = prb.chebyshev_nodes(Nz)[:, None]
    for v in s.problem.variables:
        s.set_field(v, np.zeros((Nx // 2, Nz), complex))
    s.set_field("b", 1 - z + 1e-3 * xi * z * (1 - z), "g")
    s.dz("b", "bz")
    s.step(5)
    s.sync()
    ref, floor = _reference(Nx, Nz, Ra, xi, "RK222", dt, 5, dealias=2.0)
    _check(s.get_state(), ref, floor, 1e-12)


@pytest.mark.parametrize("scheme", ["SBDF2", "SBDF4", "CNAB2"])
def test_graph_replay_matches_eager(ctx, scheme):
    """Graph replay (blocks of up to 16 steps, keyed by the step's slot in
    the multistep history ring) gives the eager steps bit for bit."""
    w = si.WORKLOADS["rb2d_64x32_rk222"]
    xi = si.rb_noise(1, w.n_z, w.n_x)
    outs = []
    for graph in (False, True):
        s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, scheme=scheme)
        s.factor(w.dt)
        s.set_initial_state(xi)
        s.step(21, graph=graph)
        s.sync()
        outs.append(s.get_state())
    assert np.array_equal(outs[0], outs[1])


# --- failure reporting (host-made failures; no GPU fault) ----------------------

def test_not_factored_dt_rejected(ctx):
    s = RBSolver(ctx, 32, 16, 1e6)
    s.factor(1e-3)
    with pytest.raises(_lib.SpectauError) as e:
        s.step(1, dt=2e-3)
    assert e.value.status == _lib.SP_ERR_NOT_FACTORED


def test_nonfinite_state_reported(ctx):
    s = RBSolver(ctx, 32, 16, 1e6)
    s.factor(1e-3)
    s.set_initial_state(si.rb_noise(2, 16, 32))
    bad = s.get_field("u")
    bad[3, 2] = np.nan
    s.set_field("u", bad)
    s.step(1)
    st, pen = ctx.sync_status()
    assert st == _lib.SP_ERR_NONFINITE and pen >= 0


def test_singular_pencil_reported(ctx):
    # without the k_x = 0 pressure gauge the mean pencil is singular
    # (the paper's reason for the ``condition`` keyword)
    from paper_1905_10388_gb300 import rb as prb
    from paper_1905_10388_gb300.solver import TauSolver
    from paper_1905_10388_gb300.tau import BCAlternative, BCSlot
    prob = prb.rb_pencil_problem(1e6)
    prob.bc_slots[5] = BCSlot([BCAlternative("w", "right")])
    s = TauSolver(ctx, prob, 32, 16, 4.0, bilinear=prb.BILINEAR_TERMS)
    s.factor(1e-3)
    st, pen = ctx.sync_status()
    assert st == _lib.SP_ERR_SINGULAR and pen == 0


def test_bad_sizes_rejected(ctx):
    with pytest.raises(_lib.SpectauError) as e:
        RBSolver(ctx, 40, 16, 1e6)           # N_gx = 60 is not 2^k or 3 2^k
    assert e.value.status == _lib.SP_ERR_ARG


@pytest.mark.parametrize("Nz", [16, 32])
def test_wide_band_two_register_window(ctx, Nz):
    """A row/variable order of the same RB pencils with kl + ku = 36 > 31
    (the back substitution keeps two window registers per lane); at N_z = 32
    the padded length 224 is not a multiple of the 64-row window."""
    from paper_1905_10388_gb300 import rb as prb
    from paper_1905_10388_gb300.solver import TauSolver
    Nx, Ra, dt, nsteps = 32, 1e5, 2e-3, 3
    V = ("w", "wz", "uz", "u", "b", "bz", "p")
    E = ("uz_def", "wz_def", "bz_def", "u", "w", "b", "div")
    s = TauSolver(ctx, prb.rb_pencil_problem(Ra, variables=V, row_order=E), Nx, Nz, 4.0, scheme="RK222",
                  bilinear=prb.BILINEAR_TERMS)
    s.state_order = prb.VARIABLES
    assert sum(s.band()[1:]) > 31
    s.factor(dt)
    xi = si.rb_noise(13, Nz, Nx)
    z = prb.chebyshev_nodes(Nz)[:, None]
    for v in s.problem.variables:
        s.set_field(v, np.zeros((s.P, Nz), complex))
    s.set_field("b", 1 - z + 1e-3 * xi * z * (1 - z), "g")
    s.dz("b", "bz")
    s.step(nsteps)
    s.sync()
    ref, floor = _reference(Nx, Nz, Ra, xi, "RK222", dt, nsteps)
    _check(s.get_state(), ref, floor, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rb_512x256_cnab2_full_size(ctx, prec):
    """CNAB2 (its CNAB1 first step, then Crank-Nicolson Adams-Bashforth) on
    the benchmarked problem: 3 steps against the oracle."""
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="CNAB2", precision=prec)
    s.factor(w.dt)
    s.set_initial_state(xi)
    s.step(3)
    s.sync()
    ref, floor = _reference(w.n_x, w.n_z, w.Ra, xi, "CNAB2", w.dt, 3, w.Pr, w.L_x)
    _check(s.get_state(), ref, floor, TOL[prec])
