"""GPU linear boundary value solve with a non-constant coefficient
(sp_solve_lbvp; Sec. "Linear boundary value solver", Sec. "Non-constant
coefficients") on the potential-vorticity inversion
dx dx psi + dz(S(z) dz psi) = q, S(z) = 1 + z + z^2/2:

* a polynomial stream function is recovered exactly (to rounding) from its
  closed-form potential vorticity, every wavenumber, k_x = 0 included;
* random potential vorticity against the FP64 oracle (dense solve per
  pencil) at 64 x 64 and 512 x 256 (the partitioned substitution), bar
  max(1e-12, 10 x the floor: the oracle's own dense-vs-SuperLU spread);
* the solve replaces the stepping factorization (stepping then asks for
  sp_factor again).
"""
import numpy as np
import scipy.sparse.linalg as spla
from numpy.polynomial import Chebyshev, Polynomial
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import lbvp as olb
from paper_1905_10388_gb300 import _lib
from paper_1905_10388_gb300.solver import Context, QGInversion
from gpu_util import record, rel_err

pytestmark = pytest.mark.gpu
S_Z = [1.0, 1.0, 0.5]                  # S(z) = 1 + z + z^2 / 2
PHI = [1.0, 0.0, -3.0, 2.0]            # phi = 2 z^3 - 3 z^2 + 1


def _cheb01(poly_z, N):
    c = Polynomial(poly_z).convert(kind=Chebyshev, domain=[0.0, 1.0]).coef
    out = np.zeros(N)
    out[: len(c)] = c
    return out


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def test_polynomial_stream_function_recovered(ctx):
    nx, nz = 32, 16
    s = QGInversion(ctx, nx, nz, _cheb01(S_Z, 3))
    P = nx // 2
    kx = 2 * np.pi * np.arange(P) / s.Lx
    phi, S = Polynomial(PHI), Polynomial(S_Z)
    q = np.zeros((P, nz), complex)
    psi = np.zeros((P, nz), complex)
    psiz = np.zeros((P, nz), complex)
    for p, k in enumerate(kx):
        amp = 1.0 if p == 0 else 0.5
        q[p] = amp * _cheb01((-k * k * phi + (S * phi.deriv()).deriv()).coef, nz)
        psi[p] = amp * _cheb01(phi.coef, nz)
        psiz[p] = amp * _cheb01(phi.deriv().coef, nz)
    X = s.invert(q)
    assert rel_err(X[0], psi) < 1e-12
    assert rel_err(X[1], psiz) < 1e-12


def _oracle(nx, nz, q):
    pr = olb.qg_problem(nz, _cheb01(S_Z, 3))
    kx = 2 * np.pi * np.arange(nx // 2) / (2 * np.pi)
    ref = olb.solve_lbvp(pr, kx, {"pv": q})
    # floor: the same systems solved by SuperLU
    alt = np.zeros_like(ref)
    for p, k in enumerate(kx):
        _, L = pr.pencil_matrices(k)
        rhs = pr.rhs_vector({"pv": q[p]}, k)
        alt[:, p, :] = spla.splu(L.tocsc()).solve(rhs).reshape(2, nz)
    return ref, [rel_err(alt[i], ref[i]) for i in range(2)]


@pytest.mark.parametrize("nx,nz", [(64, 64), (512, 256)])
def test_random_pv_matches_oracle(ctx, nx, nz):
    rng = np.random.default_rng(nx + nz)
    P = nx // 2
    q = rng.standard_normal((P, nz)) + 1j * rng.standard_normal((P, nz))
    q[0] = q[0].real
    q[:, nz // 2:] *= 1e-3                       # a resolved field: decaying spectrum
    s = QGInversion(ctx, nx, nz, _cheb01(S_Z, 3))
    X = s.invert(q)
    if nx == 512:
        assert s.spike_blocks() > 1               # the partitioned substitution
    ref, floor = _oracle(nx, nz, q)
    for i, v in enumerate(("psi", "psiz")):
        err = rel_err(X[i], ref[i])
        bar = max(1e-12, 10 * floor[i])
        record(f"lbvp_qg_{nx}x{nz}_fp64", v, err, floor[i], bar)
        assert err < bar, (v, err, floor[i])


def test_lbvp_replaces_the_stepping_factor(ctx):
    s = QGInversion(ctx, 32, 16, _cheb01(S_Z, 3))
    s.factor(1e-3)
    s.invert(np.zeros((16, 16), complex))
    with pytest.raises(_lib.SpectauError) as e:
        s.step(1)
    assert e.value.status == _lib.SP_ERR_NOT_FACTORED
