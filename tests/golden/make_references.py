"""Write the stored oracle references of the full-size parity tests.

Calls only ``oracle/`` (and the seeded input generators); nothing here comes
from the CUDA path.  Each reference is the FP64 oracle's state (or gradient)
at one of the workloads at its stated size, stored as a fixed seeded sample
of its coefficients, with the sampled norm and a rounding floor: the
relative deviation, on the same sample, of oracle variants that sum the
same arithmetic in other orders (SciPy-DCT Chebyshev sums with SuperLU in
natural column order in 2D; in 3D the largest deviation of SuperLU in
natural order, of dense LAPACK LU and of SciPy-DCT Chebyshev sums with
numpy's derivative recurrence for the initial bz).

    python tests/golden/make_references.py [--only NAME ...] [--procs N]

References (``tests/golden/ref_<name>.npz``):
  rb2d_512x256_sbdf2_1000   2D Rayleigh-Benard 512 x 256, Ra = 1e8, SBDF2,
                            dt = 1e-4, 1000 steps from seed 42; 8192
                            sampled coefficients per field
  rb3d_256x256x128_rk222_1  3D Rayleigh-Benard 256 x 256 x 128, Ra = 1e7,
                            RK222, dt = 5e-4, one step from seed 42; 64
                            sampled pencils (every field and mode)
  batch64_rk222_5           instances 0, 4, 13 and 17 of the 64-instance
                            uneven batch (seeds 1000 + i), RK222, 5 steps;
                            4096 sampled coefficients per field each
  rb2d_256x128_adjoint_500  gradient of J = 1/2 sum (b(T) - b*)^2 wrt the
                            control q at q = 0 through 500 RK222 steps
                            (256 x 128, Ra = 1e6, dt = 1e-3, noise seed 42,
                            b* the initial buoyancy of seed 43): the whole
                            scale-1 grid field
"""
import argparse
import functools
import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per process: the pool's workers (spawned, they inherit this
# environment) each take a host core, and several multi-threaded BLAS
# libraries in one process pool oversubscribe the cores many times over
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402
from oracle import rb as orb  # noqa: E402
from oracle import rb3d as orb3  # noqa: E402
from oracle import timesteppers as ots  # noqa: E402
from oracle.adjoint import RBAdjoint  # noqa: E402
from oracle.pencilwise import RungeKuttaIMEXPencilwise, problem_only  # noqa: E402

BATCH_PICKS = (0, 4, 13, 17)


def path(name):
    return os.path.join(HERE, f"ref_{name}.npz")


def sample_flat(total, count, seed):
    return np.sort(np.random.default_rng(seed).choice(total, size=min(count, total), replace=False))


def rel(a, b):
    nb = np.linalg.norm(b)
    d = np.linalg.norm(a - b)
    return float(d if nb < 1e-30 else d / nb)


def sampled(X, flat):
    S = X.shape[0]
    return X.reshape(S, -1)[:, flat]


def run_2d(nx, nz, Ra, scheme, dt, nsteps, noise, cheb="mmt", lu=None):
    sysr = orb.RB2D(nx, nz, Ra, cheb_method=cheb, lu_method=lu)
    X = sysr.initial_state(noise)
    if scheme.startswith("RK"):
        st = ots.RungeKuttaIMEX(sysr, getattr(ots, scheme))
    else:
        st = ots.SBDF(sysr, int(scheme[-1]))
    for _ in range(nsteps):
        X = st.step(X, dt)
    return X


def make_rb2d_sbdf2(procs):
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    noise = si.rb_noise(w.seed, w.n_z, w.n_x)
    nsteps = 1000
    flat = sample_flat((w.n_x // 2) * w.n_z, 8192, 2024)
    with mp.get_context("spawn").Pool(2) as pool:
        a = pool.apply_async(run_2d, (w.n_x, w.n_z, w.Ra, w.scheme, w.dt, nsteps, noise))
        b = pool.apply_async(run_2d, (w.n_x, w.n_z, w.Ra, w.scheme, w.dt, nsteps, noise, "dct", "natural"))
        X, Xv = a.get(), b.get()
    ref, var = sampled(X, flat), sampled(Xv, flat)
    floor = np.array([rel(var[i], ref[i]) for i in range(ref.shape[0])])
    np.savez_compressed(path("rb2d_512x256_sbdf2_1000"), flat=flat, ref=ref, floor=floor,
                        steps=nsteps, names=np.array(orb.RB_VARIABLES),
                        full_norm=np.linalg.norm(X.reshape(X.shape[0], -1), axis=1))


def make_rb3d(procs):
    w = si.WORKLOADS["rb3d_256x256x128_rk222"]
    noise = si.rb_noise3(w.seed, w.n_z, w.n_y, w.n_x)
    P = (w.n_x // 2) * w.n_y
    K = w.n_x // 2
    pens = np.unique(np.concatenate([[0, 1, K, K + 1, (w.n_y // 2 - 1) * K, (w.n_y - 1) * K + K - 1],
                                     sample_flat(P, 58, 2025)]))
    out = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for name, lu, cheb in (("auto", "auto", "mmt"), ("natural", "natural", "mmt"), ("dense", "dense", "mmt"),
                               ("dct", "auto", "dct")):
            sysr = orb3.RB3D(w.n_x, w.n_y, w.n_z, w.Ra, w.Pr, w.L_x, w.L_y, lu_method=lu, cheb_method=cheb)
            X = sysr.initial_state(noise)
            factory = functools.partial(problem_only, orb3.rb3d_problem, w.n_z, w.Ra, w.Pr)
            st = RungeKuttaIMEXPencilwise(sysr, ots.RK222, map_fn=pool.map, chunk=256, problem_factory=factory)
            t0 = time.time()
            X = st.step(X, w.dt)
            print(f"  3D step ({name}): {time.time() - t0:.0f} s", flush=True)
            out[name] = X[:, pens, :]
    ref = out["auto"]
    floor = np.array([max(rel(out[v][i], ref[i]) for v in ("natural", "dense", "dct")) for i in range(ref.shape[0])])
    np.savez_compressed(path("rb3d_256x256x128_rk222_1"), pencils=pens, ref=ref, floor=floor, steps=1,
                        names=np.array(orb3.RB3D_VARIABLES))


def make_batch(procs):
    ws = si.batched_workloads()
    nsteps = 5
    res = {}
    with mp.get_context("spawn").Pool(min(procs, 8)) as pool:
        jobs = {}
        for i in BATCH_PICKS:
            w = ws[i]
            noise = si.rb_noise(w.seed, w.n_z, w.n_x)
            jobs[(i, "ref")] = pool.apply_async(run_2d, (w.n_x, w.n_z, w.Ra, "RK222", w.dt, nsteps, noise))
            jobs[(i, "var")] = pool.apply_async(run_2d, (w.n_x, w.n_z, w.Ra, "RK222", w.dt, nsteps, noise,
                                                          "dct", "natural"))
        for k, j in jobs.items():
            res[k] = j.get()
    arrays = {"picks": np.array(BATCH_PICKS), "steps": nsteps, "names": np.array(orb.RB_VARIABLES)}
    for i in BATCH_PICKS:
        w = ws[i]
        flat = sample_flat((w.n_x // 2) * w.n_z, 4096, 3000 + i)
        ref, var = sampled(res[(i, "ref")], flat), sampled(res[(i, "var")], flat)
        arrays[f"flat_{i}"] = flat
        arrays[f"ref_{i}"] = ref
        arrays[f"floor_{i}"] = np.array([rel(var[f], ref[f]) for f in range(ref.shape[0])])
    np.savez_compressed(path("batch64_rk222_5"), **arrays)


def adjoint_grad(cheb, lu):
    w = si.WORKLOADS["rb2d_256x128_rk222_adjoint"]
    sysr = orb.RB2D(w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, cheb_method=cheb, lu_method=lu)
    adj = RBAdjoint(sysr)
    noise = si.rb_noise(w.seed, w.n_z, w.n_x)
    target = sysr.to_grid(adj.initial_state_q(si.rb_noise(w.seed + 1, w.n_z, w.n_x), 0.0)[sysr.var["b"]],
                          w.n_x, w.n_z)
    q = np.zeros((w.n_z, w.n_x))
    return adj.loss_and_grad(noise, target, q, w.dt, 500)


def make_adjoint(procs):
    with mp.get_context("spawn").Pool(2) as pool:
        a = pool.apply_async(adjoint_grad, ("mmt", None))
        b = pool.apply_async(adjoint_grad, ("dct", "natural"))
        (J, g), (Jv, gv) = a.get(), b.get()
    np.savez_compressed(path("rb2d_256x128_adjoint_500"), grad=g, loss=J, floor=rel(gv, g),
                        loss_floor=abs(Jv - J) / abs(J), steps=500, checkpoint=50)


MAKERS = {"rb2d_512x256_sbdf2_1000": make_rb2d_sbdf2, "rb3d_256x256x128_rk222_1": make_rb3d,
          "batch64_rk222_5": make_batch, "rb2d_256x128_adjoint_500": make_adjoint}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=list(MAKERS))
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    args = ap.parse_args()
    for name in args.only:
        t0 = time.time()
        MAKERS[name](args.procs)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
