"""Benchmark: DOF*steps/s of the IMEX spectral-tau step on GB300.

Workload (default): 2D Rayleigh-Benard, Fourier x N_x = 512 (L_x = 4) by
Chebyshev z N_z = 256, Ra = 1e8, Pr = 1, 3/2 dealiasing, SBDF2 with
dt = 1e-4, seeded synthetic initial state.  One "step" is one full IMEX
step: dealiased transforms and products of the advective RHS, right-hand
side assembly and one banded FP64 tau solve per Fourier pencil.

The headline line is the FP64 form (the paper's arithmetic throughout); the
mixed form (FP32 transforms and products, FP64 pencils) is timed in the same
run and reported beside it under "mixed".  Each form's per-field error
against the FP64 oracle (same seeded initial state, a bounded number of
steps, computed outside the timed regions) is in "error".  The ALU roofline
divides by this GPU's FP64 FMA throughput, measured at start-up.

Timing: W untimed warm-up steps and an untimed rehearsal of the K steps
(which captures their CUDA graphs), then K steps replayed from the graphs,
bracketed by a barrier and torch.cuda.synchronize() and timed with CUDA
events on the library's stream; the step's working set (factor + state,
> 129 MB) is larger than L2.  For the roofline entry the same K steps then
run launch by launch with a CUDA-event pair around every pencil solve.
Clocks are sampled with nvidia-smi over both passes.

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

import seeded_inputs as si

METRIC = "DOF·steps/s of IMEX step at stated error vs FP64 form; adjoint/forward time"
UNIT = "DOF*steps/s"
WORKLOAD = "rb2d_512x256_sbdf2"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# implicit stage solves per step of each scheme
STAGES = {"RK222": 2, "RK443": 4, "RK111": 1, "SBDF1": 1, "SBDF2": 1, "SBDF3": 1, "SBDF4": 1}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one pencil
# solve of the 512x256 SBDF2 FP64 step, summed over its eight launches
# (assembly, partitioned substitution, epilogue), from one ncu capture of
# `bench.py --precision fp64 --no-cpu-baseline --no-error --steps 3 --warmup 3`
# (metrics gpu__time_duration.sum, dram__bytes_read.sum, dram__bytes_write.sum;
# -k regex:"k_spike|k_pencil_stage_wide" -s 16 -c 8).  It is reported only
# while the kernels' sources hash to the captured ones.
SOLVE_TRAFFIC = {"workload": "rb2d_512x256_sbdf2", "precision": "fp64", "bytes": 306.3032e6,
                 "sources_sha256": "272a9c00e27801bc99b3c01e82e5e5fe76e6aac3c3de33546d1b504c131c687a"}
SOLVE_SOURCES = ("paper_1905_10388_gb300/csrc/band.cu", "paper_1905_10388_gb300/csrc/spike.cu",
                 "paper_1905_10388_gb300/csrc/internal.h", "paper_1905_10388_gb300/csrc/common.cuh",
                 "paper_1905_10388_gb300/csrc/tma.cuh")


def solve_traffic(workload, precision):
    import hashlib
    h = hashlib.sha256()
    for f in SOLVE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    t = SOLVE_TRAFFIC
    if (workload, precision, h.hexdigest()) == (t["workload"], t["precision"], t["sources_sha256"]):
        return t["bytes"]
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_rate(units_per_rank, seconds_local, world, device="cpu"):
    """Whole-job rate of `world` ranks that each processed `units_per_rank`:
    the units of all ranks divided by the slowest rank's time (all-reduce MAX
    over the process group; identity for one rank).  Returns (rate, seconds)."""
    t = float(seconds_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def solve_flops_bytes(s):
    """Algorithmic FP64 flops and bytes of one pencil-solve launch.

    Per pencil and per real right-hand side (real and imaginary parts share
    the real factor): the substitution's multiply-adds per row as the
    library reports them (sp_get_solve_work: kl forward plus kl + ku back
    for the window kernel, which multiplies every band entry; kl plus the
    listed U entries for the lane kernel, which skips the band's structural
    zeros) and one multiply by 1/U_jj; plus the right-hand-side assembly
    (one CSR matvec with the pattern's nnz, the combination of stored
    vectors) and the epilogue matvec M~ X~.
    Bytes: the stored factor as the kernel reads it plus the vectors read
    and written, all FP64.
    """
    n, kl, ku = s.band()
    fma_row, factor_pencil = s.solve_work()
    P = s.P
    M1 = s.assembly["M"][1] if "M" in s.assembly else s.assembly["values"](1, 2)[0][0]
    nnz_M = int(np.count_nonzero(M1))
    ne = len(s.nl_eqs)
    solve = 2 * fma_row * n + n                        # per real RHS
    flops = P * 2 * solve + P * 2 * 2 * nnz_M          # + epilogue M~ X~ (complex vector)
    flops += P * 2 * 2 * 3 * n                         # prologue combination of 2 vectors + F rows
    factor_bytes = P * factor_pencil
    vec_bytes = P * n * 16 * 5                         # 2 stored vectors in, X~, X, M~X~ out
    vec_bytes += P * nnz_M * 8 + ne * P * s.Nz * 16 * 2  # M~ values, two F coefficient arrays
    return flops, factor_bytes + vec_bytes


def _make_solver(ctx, w, precision, rank, z_transform=None):
    from paper_1905_10388_gb300.solver import FisherKPPSolver, RB3DSolver, RBSolver
    if isinstance(w, si.FisherWorkload):
        s = FisherKPPSolver(ctx, w.n_x, w.n_z, w.D, w.R, w.L_x, scheme=w.scheme, precision=precision)
        xi = si.fisher_noise(w.seed + rank, w.n_z, w.n_x)
    elif w.n_y > 1:
        s = RB3DSolver(ctx, w.n_x, w.n_y, w.n_z, w.Ra, w.Pr, w.L_x, w.L_y, scheme=w.scheme, precision=precision)
        xi = si.rb_noise3(w.seed + rank, w.n_z, w.n_y, w.n_x)
    else:
        s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme=w.scheme, precision=precision)
        xi = si.rb_noise(w.seed + rank, w.n_z, w.n_x)
    if z_transform:
        s.set_z_transform(z_transform)
    s.factor(w.dt)
    s.set_initial_state(xi)
    return s, xi


def _time_form(s, args, stages, stream, distributed):
    """Warm-up, graph rehearsal, the K timed steps replayed from graphs, then
    the same K steps launched one by one with events around every solve."""
    import torch
    s.step(args.warmup)
    # a rehearsal of the timed steps captures the CUDA graphs they replay
    # (blocks of up to 16 steps) outside the timed region
    s.step(args.steps, graph=True)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if distributed:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(args.steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    if distributed:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    s.set_timing(args.steps * stages)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(args.steps, graph=False)
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)
    s.sync()
    solve_ms, solve_launches = s.solve_time()
    s.set_timing(0)
    return ms, eager_ms, solve_ms, solve_launches


# Steps of the per-field error check (from the seeded initial state, GPU
# against the FP64 oracle): about 10 s of oracle work per workload size.
def error_steps(w):
    return 50 if w.dof <= 1_000_000 else 5


def oracle_states(w, xi, nsteps):
    """The FP64 oracle's state after `nsteps` steps from the seeded initial state."""
    from oracle import timesteppers as ots
    if isinstance(w, si.FisherWorkload):
        from oracle import fisher as ofk
        sysr = ofk.FisherKPP(w.n_x, w.n_z, w.D, w.R, w.L_x)
    else:
        from oracle import rb as orb
        sysr = orb.RB2D(w.n_x, w.n_z, w.Ra, w.Pr, w.L_x)
    X = sysr.initial_state(xi)
    if w.scheme.startswith("RK"):
        st = ots.RungeKuttaIMEX(sysr, getattr(ots, w.scheme))
    else:
        st = ots.SBDF(sysr, int(w.scheme[-1]))
    for _ in range(nsteps):
        X = st.step(X, w.dt)
    return X


def field_errors(s, X_ref, xi, nsteps):
    """Per-field ||x_gpu - x_ref|| / ||x_ref|| (absolute below a reference norm
    of 1e-30) over the coefficients after `nsteps` steps from `xi`."""
    s.set_initial_state(xi)
    s.step(nsteps, graph=True)
    s.sync()
    got = s.get_state()
    out = {}
    for i, name in enumerate(s.state_order):
        nr = float(np.linalg.norm(X_ref[i]))
        d = float(np.linalg.norm(got[i] - X_ref[i]))
        out[name] = d if nr < 1e-30 else d / nr
    return out


def z_path_times(local, w, rank, stream, nsteps=6):
    """3D mixed form: ms per step with the Chebyshev backward transform as the
    FFT-based DCT and as the tensor-core matrix product, each on a solver and
    context of its own (CUDA-graph steps after a rehearsal; outside every
    timed region)."""
    import torch
    from paper_1905_10388_gb300.solver import Context
    out = {}
    for kind in ("fft", "mma"):
        c = Context(local, stream.cuda_stream)
        try:
            s, _ = _make_solver(c, w, "mixed", rank, z_transform=kind)
            s.step(nsteps, graph=True)
            s.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(nsteps, graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            out[f"{kind}_ms_per_step"] = e0.elapsed_time(e1) / nsteps
        finally:
            c.close()
    out["faster"] = min(("fft", "mma"), key=lambda k: out[f"{k}_ms_per_step"])
    out["steps"] = nsteps
    return out


def stored_3d_errors(s, xi):
    """Per-field error of one step from the seeded state against the stored
    FP64 oracle reference of the 3D workload (written by
    tests/golden/make_references.py from the oracle alone), on its sampled
    pencils; None when that file is absent."""
    path = os.path.join(ROOT, "tests", "golden", "ref_rb3d_256x256x128_rk222_1.npz")
    if not os.path.exists(path):
        return None
    R = np.load(path)
    s.set_initial_state(xi)
    s.step(1)
    s.sync()
    got = s.get_state()[:, R["pencils"], :]
    out = {}
    for i, name in enumerate(R["names"]):
        nr = float(np.linalg.norm(R["ref"][i]))
        d = float(np.linalg.norm(got[i] - R["ref"][i]))
        out[str(name)] = d if nr < 1e-30 else d / nr
    return out


def run_ours(args):
    import torch
    distributed = int(os.environ.get("WORLD_SIZE", "1")) > 1
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if distributed:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1905_10388_gb300 import _lib
    from paper_1905_10388_gb300.solver import Context
    w = si.WORKLOADS[args.workload]
    fisher = isinstance(w, si.FisherWorkload)
    # measured FMA throughput of this GPU: the ALU roofline's denominators
    fp64_peak = _lib.measure_fma_peak(local, "fp64")
    fp32_peak = _lib.measure_fma_peak(local, "fp32")
    ctx = Context(local, torch.cuda.current_stream(local).cuda_stream)
    stages = STAGES.get(w.scheme, 1)
    stream = torch.cuda.current_stream(local)
    # the headline form (FP64 throughout, the paper's arithmetic, unless
    # --precision picks one) and, by default, the mixed form beside it
    forms = [args.precision] if args.precision != "both" else ["fp64", "mixed"]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    timed = {}
    solvers = {}
    for prec in forms:
        zt = args.z_transform if (prec == "mixed" and args.z_transform != "auto") else None
        s, xi = _make_solver(ctx, w, prec, rank, z_transform=zt)
        timed[prec] = _time_form(s, args, stages, stream, distributed)
        solvers[prec] = s
    clk = clocks.stop()
    head = forms[0]
    s = solvers[head]
    ms, eager_ms, solve_ms, solve_launches = timed[head]
    value, secs = job_rate(w.dof * args.steps, ms * 1e-3, world, device="cuda")
    ms = secs * 1e3

    # end to end through the public API with host buffers: upload the state,
    # K steps each followed by a device-to-host read of the first field (b or u)
    X0 = s.get_state()
    host_state = [np.ascontiguousarray(X0[i]) for i in range(s.S)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(host_state)
    probe = "u" if fisher else "b"              # the step's result read back every step
    for _ in range(args.steps):
        s.step(1)
        _ = s.get_field(probe)
    torch.cuda.synchronize()
    e2e_rate, _ = job_rate(w.dof * args.steps, time.perf_counter() - t0, world, device="cuda")
    state_bytes = s.S * s.P * s.Nz * 16
    e2e = {"value": e2e_rate, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / args.steps, "d2h_bytes_per_step": s.P * s.Nz * 16}

    # per-field error against the FP64 oracle (outside every timed region)
    errors = {}
    err_steps = None
    err_vs = "FP64 oracle, same seeded initial state"
    if rank == 0 and w.n_y == 1 and not args.no_error:
        err_steps = error_steps(w)
        X_ref = oracle_states(w, xi, err_steps)
        for prec in forms:
            errors[prec] = field_errors(solvers[prec], X_ref, xi, err_steps)
    elif rank == 0 and args.workload == "rb3d_256x256x128_rk222" and not args.no_error:
        err_steps = 1
        err_vs = "stored FP64 oracle reference of one step from the same seeded state, 64 sampled pencils"
        for prec in forms:
            e = stored_3d_errors(solvers[prec], xi)
            if e is not None:
                errors[prec] = e
    z_paths = None
    if rank == 0 and w.n_y > 1 and "mixed" in forms and not args.no_z_compare:
        z_paths = dict({"timed_path": solvers["mixed"].z_transform()},
                       **z_path_times(local, w, rank, stream))

    flops, nbytes = solve_flops_bytes(s)
    n_, kl_, ku_ = s.band()
    # the library's automatic choice of substitution kernel (sp_set_solve_kernel):
    # lane substitution (assembly, lanes, epilogue: three launches), the
    # partitioned substitution (assembly, two forward passes and their
    # recurrence, two backward passes and theirs, epilogue: eight launches),
    # or the single window kernel
    lanes = s.P >= 4096 and (kl_, kl_ + ku_) in ((9, 38), (7, 29))
    nblk = s.spike_blocks()
    factor_mb = s.P * s.solve_work()[1] / 1e6
    achieved = flops / (solve_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    if lanes:
        kernel, solve_launches_per = "k_pencil_stage<1> + k_pencil_lanes + k_pencil_stage<2>", 3
    elif nblk > 0:
        kernel = (f"partitioned substitution, {nblk} row blocks per pencil: k_pencil_stage_wide<1> + "
                  "k_spike_fwd<1> + k_spike_fwd_rec + k_spike_fwd<2> + k_spike_bwd<1> + k_spike_bwd_rec + "
                  "k_spike_bwd<2> + k_pencil_stage_wide<2>")
        solve_launches_per = 8
    else:
        kernel, solve_launches_per = "k_pencil_solve", 1
    roof = {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "traffic": solve_traffic(args.workload, head), "algorithmic_bytes": nbytes,
            "peak_source": "measured: FP64 FMA throughput of this GPU (sp_measure_fma_peak, independent "
                           "chains on every SM, best of 3); of measured",
            "ms_per_launch": solve_ms, "launches": solve_launches,
            "hbm_achieved_gbs": nbytes / (solve_ms * 1e-3) / 1e9,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "hbm_frac": nbytes / (solve_ms * 1e-3) / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
            "measured_peaks_tflops": {"fp64_fma": fp64_peak, "fp32_fma": fp32_peak}}
    launches = stages * ((5 if w.n_y > 1 else 3) + solve_launches_per) * args.steps
    result = None
    if rank == 0:
        dtype = {"fp64": "f64", "mixed": "f32+f64"}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": dtype[head],
            "data": "synthetic (seeded %s initial state)" % ("Fisher-KPP" if fisher else "Rayleigh-Benard"),
            "config": dict({"workload": args.workload, "n_x": w.n_x, "n_y": w.n_y, "n_z": w.n_z},
                           **({"D": w.D, "R": w.R} if fisher else {"Ra": w.Ra, "Pr": w.Pr}),
                           **{"scheme": w.scheme, "dt": w.dt, "dof": w.dof, "precision": head,
                              "parallelism": f"replicas{world}",
                              "l2": (f"working set > L2 (factor {factor_mb:.0f} MB read every solve)"
                                     if factor_mb > 129 else
                                     f"L2-resident (factor {factor_mb:.0f} MB < 129 MB L2; no flush)")}),
            "error": ({"vs": err_vs, "steps": err_steps,
                       "norm": "per field ||x_gpu - x_ref||_2 / ||x_ref||_2 over the coefficients",
                       "fields": errors.get(head), "max": max(errors[head].values())}
                      if head in errors else None),
            "roofline": roof, "e2e": e2e,
            "timing": {"value": "CUDA-graph replay of the steps (blocks of up to 16), inputs resident",
                       "roofline": "an eager pass of the same steps right after, CUDA events around every solve",
                       "eager_ms_per_step": eager_ms / args.steps},
            "gpu_launches": launches * len(forms),
            "clocks": clk,
        }
        if z_paths is not None:
            result["z_backward"] = z_paths
        for prec in forms[1:]:
            ms2, eager2, solve2, _ = timed[prec]
            result[prec] = {
                "value": w.dof * args.steps / (ms2 * 1e-3), "unit": UNIT, "ms_per_step": ms2 / args.steps,
                "dtype": dtype[prec], "solve_ms_per_launch": solve2,
                "over_fp64": (w.dof * args.steps / (ms2 * 1e-3)) / value,
                "error": ({"steps": err_steps, "fields": errors[prec], "max": max(errors[prec].values())}
                          if prec in errors else None)}
    ctx.close()
    if distributed:
        torch.distributed.destroy_process_group()
    return result


def run_batch(args):
    """64 independent uneven 2D RB instances advanced together (RK222)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1905_10388_gb300.solver import Context, RBSolver, batch_persistent, batch_tile, step_batched
    ws = si.batched_workloads()
    ctx = Context(0, torch.cuda.current_stream(0).cuda_stream)
    solvers = []
    for w in ws:
        s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK222", precision=args.precision)
        s.factor(w.dt)
        s.set_initial_state(si.rb_noise(w.seed, w.n_z, w.n_x))
        solvers.append(s)
    step_batched(solvers, args.warmup, graph=True)
    ctx.sync_status()
    stream = torch.cuda.current_stream(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.2)
    torch.cuda.synchronize()
    e0.record(stream)
    step_batched(solvers, args.steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st, pen = ctx.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} at pencil {pen}")
    ms = e0.elapsed_time(e1)
    dof = sum(w.dof for w in ws)
    # the same steps of every instance on its own (graph replay, one problem
    # at a time), for the comparison with the batched launches
    solo_ms = 0.0
    for s in solvers:
        s.step(2, graph=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(args.steps, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        solo_ms += e0.elapsed_time(e1)
    res = {"metric": METRIC, "value": dof * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic (seeded Rayleigh-Benard initial states)",
           "config": {"workload": "rb2d_batch64_rk222", "instances": len(ws), "dof_total": dof,
                      "n_x": sorted({w.n_x for w in ws}), "n_z": sorted({w.n_z for w in ws}),
                      "precision": args.precision, "z_tile": batch_tile(solvers),
                      "persistent": batch_persistent(solvers),
                      "launch": ("one batched launch per kernel type per stage, CUDA graph; "
                                 "launch shape (per-item CTAs or persistent grids on a work queue) and z tile "
                                 "chosen by the library's autotuner"),
                      "l2": "working set > L2"},
           "solo": {"ms_per_step_sum_of_instances": solo_ms / args.steps,
                    "batched_speedup": solo_ms / ms},
           "roofline": None, "gpu_launches": 8 * args.steps, "clocks": clk}
    ctx.close()
    return res


def run_cfl(args):
    """The 512x256 RK222 step under CFL control (Sec. "Timestep
    determination"): before every step the frequency of the state on the
    dealiased grid (sp_cfl_frequency, read back to the host), the bounded and
    thresholded step (sp_cfl_dt), and a factorization only when the step
    changes.  The timed region holds all of it."""
    import torch
    torch.cuda.set_device(0)
    from paper_1905_10388_gb300.solver import CFL, Context, RBSolver
    w = si.WORKLOADS["rb2d_512x256_sbdf2"]
    ctx = Context(0, torch.cuda.current_stream(0).cuda_stream)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme="RK222", precision=args.precision)
    dt0 = 1e-4
    s.factor(dt0)
    s.set_initial_state(si.rb_noise(w.seed, w.n_z, w.n_x))
    s.step(args.warmup)
    s.sync()
    prm = dict(safety=0.5, min_dt=1e-6, max_dt=1e-3, min_change=0.5, max_change=1.5, threshold=0.1)
    ctl = CFL(s, (("u", "x"), ("w", "z")), initial_dt=dt0, **prm)
    t_cfl = []
    for _ in range(3):                        # warm the frequency path (scratch, plans)
        t0 = time.perf_counter()
        s.cfl_frequency(ctl.velocities)
        t_cfl.append(time.perf_counter() - t0)
    stream = torch.cuda.current_stream(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.2)
    torch.cuda.synchronize()
    e0.record(stream)
    ctl.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st, pen = ctx.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} at pencil {pen}")
    ms = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    for _ in range(10):
        s.cfl_frequency(ctl.velocities)
    freq_ms = (time.perf_counter() - t0) / 10 * 1e3
    res = {"metric": METRIC, "value": w.dof * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic (seeded Rayleigh-Benard initial state)",
           "config": {"workload": "rb2d_512x256_rk222_cfl", "n_x": w.n_x, "n_z": w.n_z, "Ra": w.Ra,
                      "scheme": "RK222", "precision": args.precision, "cfl": prm, "initial_dt": dt0,
                      "l2": "working set > L2 (factor read every solve)"},
           "cfl": {"factorizations": ctl.factorizations, "dt_first": ctl.history[0], "dt_last": ctl.history[-1],
                   "distinct_dt": len(set(ctl.history)), "frequency_ms": freq_ms},
           "roofline": None,
           # per step: frequency (z backward, x rows, maximum) + two RK222 stages
           # of four launches; one k_band_factor per change of step
           "gpu_launches": args.steps * (3 + 2 * 4) + ctl.factorizations, "clocks": clk}
    ctx.close()
    return res


def run_evp(args):
    """Growth rate of the mode nearest zero in every pencil of the
    linearized 512x256 Rayleigh-Benard problem at Ra = 1e4 (Sec. "Eigenvalue
    solver", shift and invert): one factorization of L~ + sigma_T M~, then
    `steps` power iterations (a banded solve and a normalization each)."""
    import torch
    torch.cuda.set_device(0)
    import scipy.linalg as sla
    from oracle import rb as orb
    from paper_1905_10388_gb300.solver import Context, RBOnsetEVP
    Nx, Nz, Ra, Lx = 512, 256, 1e4, 4.0
    ctx = Context(0, torch.cuda.current_stream(0).cuda_stream)
    e = RBOnsetEVP(ctx, Nx, Nz, Ra, L_x=Lx)
    e.growth_rates(0.0, iters=args.warmup)
    stream = torch.cuda.current_stream(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.2)
    torch.cuda.synchronize()
    e0.record(stream)
    rates = e.growth_rates(0.0, iters=args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    dof = 7 * Nx * Nz
    # oracle: the dense generalized eigensolver on two sampled pencils
    kx = 2 * np.pi * np.arange(Nx // 2) / Lx
    t0 = time.perf_counter()
    worst = 0.0
    for p in (1, 3):
        M, Lm = orb.rb_onset_pencil(Nz, Ra, 1.0, kx[p])
        w = sla.eig(-Lm.toarray(), M.toarray(), right=False)
        w = w[np.isfinite(w)]
        ref = w[np.argmin(np.abs(w))]
        worst = max(worst, abs(rates[p] - ref) / max(1.0, abs(ref)))
    t_pencil = (time.perf_counter() - t0) / 2
    res = {"metric": "pencil eigenmodes/s (mode nearest the target, every pencil)",
           "value": (Nx // 2) / (ms * 1e-3), "unit": "pencils/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (the linearized Rayleigh-Benard pencils; start vectors all ones)",
           "config": {"workload": "rb2d_512x256_onset_evp", "n_x": Nx, "n_z": Nz, "Ra": Ra, "target": 0.0,
                      "iterations": args.steps, "dof": dof, "l2": "working set > L2 (factor read every iteration)"},
           "evp": {"ms_total": ms, "max_rate": float(np.max(rates.real)), "sampled_rel_err_vs_dense": worst},
           "cpu_baseline": {"value": 1.0 / t_pencil, "unit": "pencils/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": f"dense scipy.linalg.eig of 2 pencils (n = {7 * Nz}), "
                                                         f"{t_pencil:.1f} s each"},
           "roofline": None, "gpu_launches": 1 + 2 * args.steps, "clocks": clk}
    ctx.close()
    return res


def run_adjoint(args):
    """Gradient of the final-buoyancy misfit through K RK222 steps (discrete
    adjoint with checkpoints every 50 steps): forward sweep, adjoint sweep,
    their time ratio, and the gradient checked against central differences
    of the FP64 forward loss in a random direction."""
    import torch
    torch.cuda.set_device(0)
    from paper_1905_10388_gb300.adjoint import RBAdjoint
    from paper_1905_10388_gb300.solver import Context, RBSolver
    w = si.WORKLOADS[args.workload]
    nsteps = args.steps
    ctx = Context(0, torch.cuda.current_stream(0).cuda_stream)
    stream = torch.cuda.current_stream(0)
    xi = si.rb_noise(w.seed, w.n_z, w.n_x)
    s = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme=w.scheme, precision=args.precision)
    s.factor(w.dt)
    s.set_initial_state(si.rb_noise(w.seed + 1, w.n_z, w.n_x))
    target = s.get_field("b", "g")                            # b*: the initial buoyancy of seed + 1
    adj = RBAdjoint(s, xi, target, checkpoint=50)
    q = np.zeros((w.n_z, w.n_x))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    for _ in range(max(1, args.warmup // 3)):                   # warm-up: one full gradient
        J, cps, r = adj.forward(q, nsteps)
        adj.backward(cps, r, nsteps)
    s.set_initial_state(xi)
    _, t_plain = timed(lambda: s.step(nsteps))
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.2)
    (J, cps, r), t_fwd = timed(lambda: adj.forward(q, nsteps))
    g, t_bwd = timed(lambda: adj.backward(cps, r, nsteps))
    clk = clocks.stop()
    ctx.sync_status()

    # gradient check in FP64: adjoint directional derivative vs central
    # differences (Richardson-extrapolated) of the forward loss
    s64 = RBSolver(ctx, w.n_x, w.n_z, w.Ra, w.Pr, w.L_x, scheme=w.scheme, precision="fp64")
    s64.factor(w.dt)
    a64 = RBAdjoint(s64, xi, target, checkpoint=50)
    J64, g64 = a64.loss_and_grad(q, nsteps)
    g64 = g64.cpu().numpy()
    d = np.random.default_rng(w.seed + 2).standard_normal(q.shape)

    def central(eps):
        return (a64.forward(q + eps * d, nsteps)[0] - a64.forward(q - eps * d, nsteps)[0]) / (2 * eps)

    fd = (4 * central(5e-3) - central(1e-2)) / 3
    an = float(np.sum(g64 * d))
    gm = g.cpu().numpy()
    res = {"metric": METRIC, "value": w.dof * nsteps / ((t_fwd + t_bwd) * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": nsteps, "warmup": args.warmup, "ms_per_step": (t_fwd + t_bwd) / nsteps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic (seeded Rayleigh-Benard initial state; target: initial buoyancy of seed + 1)",
           "config": {"workload": args.workload, "n_x": w.n_x, "n_z": w.n_z, "Ra": w.Ra, "scheme": w.scheme,
                      "dt": w.dt, "dof": w.dof, "precision": args.precision, "checkpoint": 50,
                      "step": "value counts forward + adjoint sweep of one gradient",
                      "l2": "working set < L2 (factor ~49 MB)"},
           "adjoint_over_forward": t_bwd / t_plain,
           "times_ms": {"forward_plain": t_plain, "forward_with_checkpoints": t_fwd, "adjoint_sweep": t_bwd},
           "gradient_check": {"fd": fd, "adjoint": an, "rel_err": abs(fd - an) / abs(fd),
                              "precision": "fp64", "mixed_vs_fp64_rel": float(
                                  np.linalg.norm(gm - g64) / np.linalg.norm(g64)), "loss": J64},
           "roofline": None, "clocks": clk}
    ctx.close()
    return res


def oracle_rate(workload, steps_timed, warm):
    """The FP64 CPU oracle on the same workload: returns (DOF*steps/s, seconds)."""
    from oracle import rb as orb
    from oracle import timesteppers as ots
    w = si.WORKLOADS[workload]
    if isinstance(w, si.FisherWorkload):
        from oracle import fisher as ofk
        sysr = ofk.FisherKPP(w.n_x, w.n_z, w.D, w.R, w.L_x)
        X = sysr.initial_state(si.fisher_noise(w.seed, w.n_z, w.n_x))
    else:
        sysr = orb.RB2D(w.n_x, w.n_z, w.Ra, w.Pr, w.L_x)
        X = sysr.initial_state(si.rb_noise(w.seed, w.n_z, w.n_x))
    st = ots.RungeKuttaIMEX(sysr, getattr(ots, w.scheme)) if w.scheme.startswith("RK") else ots.SBDF(sysr, 2)
    for _ in range(warm):
        X = st.step(X, w.dt)
    t0 = time.perf_counter()
    for _ in range(steps_timed):
        X = st.step(X, w.dt)
    dt = time.perf_counter() - t0
    return w.dof * steps_timed / dt, dt


def oracle_rate_3d(workload, sample_pencils=16):
    """The FP64 CPU oracle on the 3D workload, extrapolated from a sample: one
    full-size advective right-hand side (all transforms and products) timed
    whole, and the stage solves of `sample_pencils` pencils with their stored
    factors; a step = stages x (right-hand side + P pencil solves).
    Returns (DOF*steps/s, seconds of CPU work, description)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    from oracle import rb3d as orb3
    w = si.WORKLOADS[workload]
    sysr = orb3.RB3D(w.n_x, w.n_y, w.n_z, w.Ra, w.Pr, w.L_x, w.L_y)
    X = sysr.initial_state(si.rb_noise3(w.seed, w.n_z, w.n_y, w.n_x))
    t0 = time.perf_counter()
    sysr.nonlinear(X)
    t_rhs = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    picks = rng.choice(sysr.P, sample_pencils, replace=False)
    gamma = 1.0 - 1.0 / np.sqrt(2.0)
    t_solve = 0.0
    for p in picks:
        M, L = sysr.problem.pencil_matrices(sysr.wavenumber(int(p)))
        lu = spla.splu(sps.csc_matrix(M + w.dt * gamma * L))
        b = M @ sysr.to_pencil(X, int(p))
        t1 = time.perf_counter()
        lu.solve(b)
        t_solve += time.perf_counter() - t1
    t_solve /= sample_pencils
    stages = STAGES.get(w.scheme, 1)
    step = stages * (t_rhs + sysr.P * t_solve)
    desc = (f"extrapolated: one full-size right-hand side ({t_rhs:.1f} s) and {sample_pencils} sampled pencil "
            f"solves ({t_solve * 1e3:.2f} ms each, stored SuperLU factors); step = {stages} x (RHS + "
            f"{sysr.P} solves) = {step:.1f} s")
    return w.dof / step, t_rhs + t_solve * sample_pencils, desc


def cpu_baseline(workload, steps=2):
    if si.WORKLOADS[workload].n_y > 1:
        rate, secs, desc = oracle_rate_3d(workload)
        return {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc}
    rate, secs = oracle_rate(workload, steps, warm=2)
    return {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{steps} steps of {workload} after 2 warm-up steps (factorizations), "
                      f"{secs:.1f} s; numpy/scipy FP64, SuperLU single-threaded"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    w = si.WORKLOADS[args.workload]
    if w.n_y > 1:
        rate, secs, desc = oracle_rate_3d(args.workload)
        return {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": 1,
                "warmup": args.warmup, "ms_per_step": w.dof / rate * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": args.workload, "n_x": w.n_x, "n_y": w.n_y, "n_z": w.n_z, "scheme": w.scheme},
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    steps = max(1, min(args.steps, 3))
    rate, secs = oracle_rate(args.workload, steps, warm=max(1, min(args.warmup, 2)))
    return {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": secs / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "n_x": w.n_x, "n_z": w.n_z, "scheme": w.scheme},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{steps} steps after warm-up, {secs:.1f} s"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="default 200 (500 for the adjoint workload)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both (default): the FP64 form as the headline and the mixed form beside it")
    ap.add_argument("--no-error", action="store_true", help="skip the per-field error check against the oracle")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--z-transform", default="auto", choices=["auto", "fft", "mma"],
                    help="mixed form: Chebyshev backward path of the timed solver (default: the library's choice)")
    ap.add_argument("--no-z-compare", action="store_true",
                    help="3D: skip timing the FFT and tensor-core Chebyshev backward paths side by side")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 500 if args.workload.endswith("_adjoint") else 200
    if args.warmup < 3:
        args.warmup = 3
    if args.precision == "both" and args.workload in (
            "rb2d_batch64_rk222", "rb2d_512x256_rk222_cfl", "rb2d_512x256_onset_evp") or (
            args.precision == "both" and args.workload.endswith("_adjoint")):
        # the batched and adjoint workloads are posed in the mixed form
        # (FP32 transforms and products, FP64 pencils); CFL and EVP lines too
        args.precision = "mixed"
    if args.impl == "reference":
        res = run_reference(args)
    elif args.workload == "rb2d_batch64_rk222":
        res = run_batch(args)
    elif args.workload.endswith("_adjoint"):
        res = run_adjoint(args)
    elif args.workload == "rb2d_512x256_rk222_cfl":
        res = run_cfl(args)
    elif args.workload == "rb2d_512x256_onset_evp":
        res = run_evp(args)
    else:
        res = run_ours(args)
        if res is not None and not args.no_cpu_baseline and int(os.environ.get("WORLD_SIZE", "1")) == 1:
            res["cpu_baseline"] = cpu_baseline(args.workload)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
