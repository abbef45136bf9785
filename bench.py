"""Throughput of one full CDI + NS time step (4 RK stages, 4 pressure solves to
a 1e-8 relative residual) on the largest single-GPU workload: the wide 3D drop,
512x256x256 cells on [0,2]x[0,1]x[0,1], density ratio 20, spreading on a 45 deg
wall, FP32-mixed (FP32 state and stencils, FP64 reductions, double-float
defect correction), first guess of every solve from the previous pressure,
through the libcdi C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints ONE JSON line on rank 0.  The GPU arm runs W warm-up steps and times K
steps with CUDA events on the library's stream; every field of the workload
(134 MB each) is larger than the 129 MB L2, so no flush is needed between
steps.  `value` is whole-job Mcell-steps/s.  `e2e` is the same metric when
every step uploads the state from pinned host memory and reads every field
back.  `forms` adds the 512x128 two-phase Couette in FP64 (the parity form)
and FP32-mixed, the batched sweep, the 256^3 drop and the learned first guess.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores.  With N > 1 GPUs the workload is replicated, one independent replica
per rank (the single grid does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s per full CDI+NS step, learned/batched vs plain, same accuracy"
UNIT = "Mcell-steps/s"
WORKLOAD = "drop3d_512x256x256_fp32mixed"
PRESSURE_TOL = 1e-8
# finest-level sweeps V(1,1) and V(2,2) on the separately launched levels below it: measured
# fastest a step on this workload once the pressure solve ran as one graph (V(1,2) with the
# finest level's counts everywhere, the library's 3D default, is 13 % slower here)
SMOOTHING_3D = (1, 1)
COARSE_SMOOTHING_3D = (2, 2)
SMOOTHING_2D = (1, 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    return ap.parse_args()


def workload(nx=512):
    """The wide 3D drop at nx x nx/2 x nx/2 (nx = 512: the bench workload)."""
    from paper_2412_16843_gb300 import inputs
    return inputs.drop_3d_wide(nx)


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of the kernels the roofline can name
# (unique words each launch must read or write at least once)
# ---------------------------------------------------------------------------
def vcycle_words(D, sweeps=4):
    """Words per finest-level cell of one V-cycle (the per-unit figure of the
    measurement contract): on the finest level `sweeps` smoothing sweeps x 4
    words (p read and write, f, phi; the contract's V(2,2) cycle has 4), the
    residual 4, the restriction 1 + 2^-D, the prolongation and correction
    2 + 2^-D; the whole hierarchy weighs 1/(1 - 2^-D) of the finest level
    (with 4 sweeps about 31 words in 2D, 27 in 3D)."""
    fine = sweeps * 4 + 4 + (1 + 2.0 ** -D) + (2 + 2.0 ** -D)
    return fine / (1 - 2.0 ** -D)


def step_bytes(D, N, word, vcycles_per_step, sweeps=4):
    """Algorithmic bytes of one full step, B = W [4 * 5(1+D) + 4 ((D+1) + (2D+1)
    + N_V V_D)] per cell: per RK stage the fused stencil minimum (read the stage
    state and y^n, read+write the accumulator, write the next stage: 5(1+D)
    words), per pressure solve the divergence (D velocity components read, f
    written: D+1 words), the projection (2D+1) and N_V V-cycles of V_D words
    (V_D with the cycle's own number of finest-level sweeps); W is the state
    word size."""
    nv_per_solve = vcycles_per_step / 4.0
    words = 4 * 5 * (1 + D) + 4 * ((D + 1) + (2 * D + 1) + nv_per_solve * vcycle_words(D, sweeps))
    return N * word * words


def onepass_sweep_words(sweeps):
    """FP32 words a cell of one launch of the 3D one-pass finest-level sweep,
    averaged over the launches of one V-cycle with `sweeps` sweeps: the first
    reads rho and r and writes e (3), the plain ones also read the old e (4),
    the last one reads rho, r and the old e and reads and writes the
    double-float p instead of writing e (3 + 4)."""
    return (3 + 4 * (sweeps - 2) + 7) / sweeps


def algorithmic_bytes(kernel, dim, N, NP, word, sweeps=3):
    D = dim
    words = {
        # 3D: one-pass sweeps (both colours a launch); 2D: one colour a launch (rho, the other
        # colour's e, own r, own e written)
        "rbgs0": onepass_sweep_words(sweeps) * N if D == 3 else 2.5 * N,
        # double-float residual: p (2 FP32 words), f, the densities the coefficients come from, r written
        "resid": 5 * N,
        "mom": (3 * D + 2) * N + NP,                           # u, m, phi, mu_c in; rhs of every component out
        "phi_rhs": (3 * D + 2) * N + NP,                       # phi, u, n in; rhs_phi, m out
        "cell": (3 + D) * N,                                   # phi, psi in; n, mu_c out
        "psi": 2 * N,
        "stage_mom": (2 + 5 * D) * N,
    }[kernel]
    if kernel in ("rbgs0", "resid"):
        return words * 4  # FP32 words in every precision
    return words * word


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (the summary stores the source hash)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get(kernel)
    if not ent:
        return None
    h = hashlib.sha256()
    for rel in ent["sources"]:
        src = os.path.join(ROOT, rel)
        if not os.path.exists(src):
            return None
        with open(src, "rb") as f:
            h.update(f.read())
    return ent["dram_bytes_per_launch"] if h.hexdigest()[:16] == ent["sources_sha256_16"] else None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_NX = 128   # the wide drop at 128 x 64 x 64 (h = 1/64): about 25 s a step on one core


def _oracle_worker(nx, steps, warmup, q):
    """One oracle replica: `warmup` untimed and `steps` timed steps of the wide
    drop at nx x nx/2 x nx/2 (run in a spawned process)."""
    sys.path.insert(0, ROOT)
    import oracle
    wl = workload(nx)
    o = oracle.from_workload(wl, tol=PRESSURE_TOL)
    if warmup:
        o.step(wl.dt, warmup)
    t0 = time.perf_counter()
    o.step(wl.dt, steps)
    q.put((wl.cells * steps, time.perf_counter() - t0))


def oracle_rate(nx, steps, warmup=0, procs=1):
    """Mcell-steps/s of the FP64 oracle as it stands (single-threaded code):
    `procs` independent replicas of the same sample run at once, one per host
    core, and the rate is all their cell-steps over the slowest one's time.
    Processes are spawned (no fork after CUDA use)."""
    import multiprocessing as mpr
    ctx = mpr.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(nx, steps, warmup, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    res = [q.get() for _ in ps]
    for p in ps:
        p.join()
    units = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return units / slowest / 1e6, slowest


def cpu_baseline_report():
    """The oracle on the bench workload's set-up at 128 x 64 x 64 (1/64 of the
    cells, the same domain, fluids, wall and initial drop): one step from the
    initial state, on one core and on every host core (one replica per core)."""
    cores = os.cpu_count() or 1
    v1, t1 = oracle_rate(ORACLE_SAMPLE_NX, 1)
    vn, tn = oracle_rate(ORACLE_SAMPLE_NX, 1, procs=cores)
    n = ORACLE_SAMPLE_NX
    sample = ("one step from the initial state of the bench workload's set-up at %dx%dx%d cells "
              "(h = 2/%d), %.1f s on one core; all cores: %d replicas at once, %.1f s"
              % (n, n // 2, n // 2, n, t1, cores, tn))
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_core_value": v1}


def job_rate(units_per_rank, local_seconds, world, device):
    """Whole-job rate of `world` replicas: the units all ranks processed over
    the slowest rank's time (max over ranks, an all-reduce where world > 1).
    Returns (rate in units per second, slowest seconds)."""
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    slowest = float(t.item())
    return units_per_rank * world / slowest, slowest


def reference_arm(args, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # one untimed step per candidate grid sizes the sample so the whole
    # warm-up + timed run ends within a few minutes
    budget = 150.0
    nx = ORACLE_SAMPLE_NX
    while nx > 32:
        _, t = oracle_rate(nx, 1)
        if (args.steps + args.warmup) * t <= budget:
            break
        nx //= 2
    value, secs = oracle_rate(nx, args.steps, warmup=args.warmup, procs=cores)
    sample = ("the bench workload's set-up at %dx%dx%d cells, %d warm-up and %d timed steps per replica, "
              "%d replicas (one per host core)" % (nx, nx // 2, nx // 2, args.warmup, args.steps, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "pressure_tol": PRESSURE_TOL,
                                        "sample_grid": [nx, nx // 2, nx // 2]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
ROOF_KERNELS = ("rbgs0", "resid", "mom")
# the other kernel classes of the step, timed the same way (time per step; bytes where the
# per-launch count is defined above)
BREAKDOWN_KERNELS = ("resid_restrict0", "prolong0", "rbgs", "coarse", "phi_rhs", "cell", "psi", "wall",
                     "stage_phi", "stage_mom", "div", "project")


def kernel_rooflines(s, wl, hbm, steps=2, classes=ROOF_KERNELS):
    """Per-launch device time of the largest kernels of the step (launch
    profiler: CUDA events on the library's stream around each launch; the
    pressure solve then runs without its graphs) over `steps` steps, against
    each kernel's algorithmic bytes where that is defined."""
    import torch
    out = {}
    for kc in classes:
        s.profile_start(kc, 1 << 14)
        s.step(wl.dt, steps)
        torch.cuda.synchronize()
        ms, n = s.profile_stop()
        if not n:
            continue
        avg = ms / n / 1e3
        out[kc] = {"launches": n, "avg_launch_us": avg * 1e6, "ms_per_step": ms / steps}
        try:
            nbytes = algorithmic_bytes(kc, wl.dim, wl.cells, wl.n[0] * wl.n[1], 4, sum(SMOOTHING_3D))
        except KeyError:
            continue
        out[kc].update({"algorithmic_bytes_per_launch": nbytes, "achieved": nbytes / avg / 1e9,
                        "frac": nbytes / avg / 1e9 / hbm})
    return out


def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2412_16843_gb300 import build, cdi

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    wl = workload()
    s = cdi.from_workload(wl, precision=cdi.FP32_MIXED, tol=PRESSURE_TOL, max_vcycles=100)
    s.set_exec(cdi.EXEC_KERNELS)
    s.set_solver(PRESSURE_TOL, 100, cdi.WARM_PREV)
    s.set_smoothing(*SMOOTHING_3D)
    s.set_coarse_smoothing(*COARSE_SMOOTHING_3D)
    stream = s.stream

    s.step(wl.dt, args.warmup)
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches = 0
    cyc = []
    for k in range(args.steps):
        starts[k].record(stream)
        s.step(wl.dt, 1)
        ends[k].record(stream)
        launches += s.launches_per_step()
        cyc.append(s.last_stats()["total_cycles_call"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = sum(step_ms)
    clk = clocks.stop()

    rate, slowest_s = job_rate(wl.cells * args.steps, ms / 1e3, world, "cuda")
    ms_max = slowest_s * 1e3
    value = rate / 1e6

    # end to end through the public API with host buffers
    ne = args.e2e_steps
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_h = pin(s.cell_shape)
    vel_h = [pin(s.face_shape(a)) for a in range(s.dim)]
    p_h = pin(s.cell_shape)
    s.get_fields((phi_h, vel_h, p_h))
    h2d = phi_h.nbytes + sum(v.nbytes for v in vel_h)
    d2h = phi_h.nbytes + sum(v.nbytes for v in vel_h) + p_h.nbytes
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(ne):
        s.set_state(phi_h, vel_h)
        s.step(wl.dt, 1)
        s.get_fields((phi_h, vel_h, p_h))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = job_rate(wl.cells * ne, e2e_s, world, "cuda")[0] / 1e6

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    # the contract's algorithmic bytes of every timed step with its own V-cycle count
    nbytes = sum(step_bytes(wl.dim, wl.cells, 4, c, sum(SMOOTHING_3D)) for c in cyc)
    achieved = nbytes / (ms / 1e3) / 1e9
    per_kernel = kernel_rooflines(s, wl, hbm)
    breakdown = kernel_rooflines(s, wl, hbm, classes=BREAKDOWN_KERNELS)
    roof = {"bound": "hbm", "kernel": "step", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic_for("step_wide"), "peak_source": peak_kind,
            "algorithmic_bytes_per_step": nbytes / args.steps, "avg_step_ms": ms / args.steps,
            "what": "one full step (all its launches) timed with CUDA events on the library's stream; "
                    "bytes from the per-cell formula with each timed step's own V-cycle count and the "
                    "cycle's %d finest-level sweeps" % sum(SMOOTHING_3D),
            "kernels": per_kernel, "other_kernels": breakdown}
    del s
    torch.cuda.empty_cache()
    forms = None
    if not args.no_forms and world == 1:
        forms = forms_report()
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_report()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(wl.n), "cells": wl.cells, "dt": wl.dt,
                   "precision": "fp32_mixed (FP32 state and stencils, FP64 reductions, double-float "
                                "defect correction, FP64 coarsest solve)",
                   "pressure_tol": PRESSURE_TOL, "vcycles_per_step": float(np.mean(cyc)),
                   "vcycles_per_step_min_max": [int(min(cyc)), int(max(cyc))],
                   "exec": "kernels", "warm_start": "previous pressure",
                   "smoothing": "V(%d,%d), V(%d,%d) on the separately launched coarser levels"
                                % (SMOOTHING_3D + COARSE_SMOOTHING_3D),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "not flushed: every field (134 MB) is larger than the 129 MB L2"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": ne},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)


def _timed_steps(step_fn, nsteps, flush):
    """Device time (ms) of nsteps calls of step_fn, each after an L2 flush."""
    import torch
    total = 0.0
    for k in range(nsteps):
        flush.fill_(k & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        step_fn()
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    return total


UNET_FLOPS_PER_VOXEL = sum(2 * t * ci * co / 8 ** lvl for (_, ci, co, t), lvl in
                           zip((("e0", 2, 16, 27), ("e1", 16, 32, 27), ("e2", 32, 64, 27), ("b", 64, 128, 27),
                                ("d2", 192, 64, 27), ("d1", 96, 32, 27), ("d0", 48, 16, 27), ("head", 16, 1, 1)),
                               (0, 1, 2, 3, 2, 1, 0, 0)))


def unet_form(flush, n_train=64, pairs=40, iters=800, n_infer=256):
    """Learned first guess: pairs from the first steps of an n_train^3 drop,
    Adam on the GPU, then V-cycles per solve and time per step from zero, from
    the previous pressure and from the network; and the device time of one
    forward pass at n_infer^3 against the dense BF16 peak."""
    import numpy as np
    import torch

    from paper_2412_16843_gb300 import cdi, inputs
    wl = inputs.drop_3d(n_train)
    dt = inputs.stable_dt(wl)
    s = cdi.from_workload(wl, precision=cdi.FP64, tol=PRESSURE_TOL)
    X, T = [], []
    for _ in range(pairs):
        s.step(dt, 1)
        f, p = s.last_pressure()
        x, t = inputs.unet_pair(f, p, s.get_fields()[0], wl.rho1, wl.rho2, wl.h)
        X.append(x)
        T.append(t)
    phi, vel, _ = s.get_fields()
    del s
    net = cdi.Unet((n_train,) * 3)
    net.set_params(inputs.unet_initial_params(0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = [net.train_step(X[i % pairs], T[i % pairs], lr=1e-3 if i < 0.6 * iters else 3e-4)
              for i in range(iters)]
    train_s = time.perf_counter() - t0
    res = {"grid": n_train, "pairs": pairs, "adam_steps": iters, "train_ms_per_step": 1e3 * train_s / iters,
           "loss_first": float(np.mean(losses[:pairs])), "loss_last": float(np.mean(losses[-pairs:])),
           "pressure_tol": PRESSURE_TOL, "exec": "kernels"}
    for name, warm in (("zero", cdi.WARM_ZERO), ("previous", cdi.WARM_PREV), ("network", cdi.WARM_UNET)):
        r = cdi.from_workload(wl, precision=cdi.FP64, tol=PRESSURE_TOL)
        r.set_exec(cdi.EXEC_KERNELS)
        r.set_solver(PRESSURE_TOL, 100, warm)
        if warm == cdi.WARM_UNET:
            r.set_warm_unet(net)
        r.set_state(phi, vel)
        cyc = 0
        ms = 0.0
        for _ in range(8):
            ms += _timed_steps(lambda: r.step(dt, 1), 1, flush)
            cyc += r.last_stats()["total_cycles_call"]
        res["vcycles_per_solve_" + name] = cyc / 32.0
        res["ms_per_step_" + name] = ms / 8
        del r
    params = net.get_params()
    del net
    torch.cuda.empty_cache()
    # the wide 3D drop (512 x 256 x 256, density ratio 20): V-cycles per solve and time per step
    # from zero, from the previous pressure and from the network trained above (it is fully
    # convolutional); warm-up steps first, then timed steps, each mode from the same initial state
    wl5 = inputs.drop_3d_wide(512)
    c5 = {"grid": list(wl5.n), "warmup_steps": 10, "timed_steps": 10, "dt": wl5.dt, "precision": "fp32_mixed",
          "exec": "kernels", "pressure_tol": PRESSURE_TOL}
    for name, warm in (("zero", cdi.WARM_ZERO), ("previous", cdi.WARM_PREV), ("network", cdi.WARM_UNET)):
        r = cdi.from_workload(wl5, precision=cdi.FP32_MIXED, tol=PRESSURE_TOL)
        r.set_exec(cdi.EXEC_KERNELS)
        r.set_solver(PRESSURE_TOL, 100, warm)
        big = None
        if warm == cdi.WARM_UNET:
            big = cdi.Unet(wl5.n)
            big.set_params(params)
            r.set_warm_unet(big)
        r.step(wl5.dt, 10)
        cyc, ms = 0, 0.0
        for _ in range(10):
            ms += _timed_steps(lambda: r.step(wl5.dt, 1), 1, flush)
            cyc += r.last_stats()["total_cycles_call"]
        c5["vcycles_per_solve_" + name] = cyc / 40.0
        c5["ms_per_step_" + name] = ms / 10
        del r, big
        torch.cuda.empty_cache()
    res["drop3d_512x256x256"] = c5
    big = cdi.Unet((n_infer,) * 3)
    big.set_params(params)
    N = n_infer ** 3
    x = torch.randn(N * 2, dtype=torch.float32, device="cuda")
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(big.stream):
        for _ in range(2):
            big.forward_device(x, y)
    ms = _timed_steps(lambda: big.forward_device(x, y), 5, flush) / 5
    flops = UNET_FLOPS_PER_VOXEL * N
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peak = json.load(f).get("bf16_tflops")
    res["inference"] = {"grid": n_infer, "ms": ms, "flops": flops, "tflops": flops / ms / 1e9,
                        "bf16_peak_tflops": peak, "frac": flops / ms / 1e9 / peak if peak else None,
                        "peak_source": "measured (burst)"}
    del big
    torch.cuda.empty_cache()
    return res


def forms_report(steps=30):
    """The other forms on their own workloads (one GPU): the 512x128 two-phase
    Couette in FP64 (the parity form; persistent step kernel, L2-resident) and
    FP32-mixed, the batched sweep of 512 uneven 2D instances against looping
    the single-grid step over the same instances, the 3D 256^3 drop, and the
    learned first guess."""
    import numpy as np
    import torch

    from paper_2412_16843_gb300 import cdi, inputs
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hbm, peak_kind = peaks()
    out = {}
    # Couette 512x128 in FP64 and FP32-mixed (L2-resident: a 256 MiB write flushes L2 before each step)
    wl = inputs.couette_2d(512, 128, 1.0)
    for name, prec in (("fp64_couette2d_512x128", cdi.FP64), ("fp32_mixed_couette2d_512x128", cdi.FP32_MIXED)):
        s = cdi.from_workload(wl, precision=prec, tol=PRESSURE_TOL)
        s.set_exec(cdi.EXEC_PERSISTENT)
        s.set_solver(PRESSURE_TOL, 100, cdi.WARM_EXTRAP)
        s.step(wl.dt, 3)
        cyc = 0
        s.profile_start("step", 1 << 12)

        def one():
            nonlocal cyc
            s.step(wl.dt, 1)
            cyc += s.last_stats()["total_cycles_call"]
        ms = _timed_steps(one, steps, flush)
        kms, kn = s.profile_stop()
        word = 8 if prec == cdi.FP64 else 4
        nbytes = step_bytes(2, wl.cells, word, cyc / steps, sum(SMOOTHING_2D))
        ach = nbytes / (kms / max(kn, 1) / 1e3) / 1e9
        out[name] = {"value": wl.cells * steps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps,
                     "pressure_tol": PRESSURE_TOL, "vcycles_per_step": cyc / steps, "exec": "persistent",
                     "warm_start": "extrapolated", "l2_resident": True,
                     "roofline": {"bound": "hbm", "kernel": "step", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                  "frac": ach / hbm, "peak_source": peak_kind,
                                  "traffic": traffic_for("step") if prec == cdi.FP64 else None,
                                  "algorithmic_bytes_per_launch": nbytes,
                                  "note": "L2-resident: the HBM fraction is not the bound here"}}
        del s
    # batched sweep vs looping the single-grid step
    wls = inputs.sweep_2d()
    cells = sum(w.cells for w in wls)
    solvers = []
    for w in wls:
        sv = cdi.from_workload(w, precision=cdi.FP32_MIXED, tol=PRESSURE_TOL)
        sv.set_solver(PRESSURE_TOL, 100, cdi.WARM_EXTRAP)
        sv.set_smoothing(2, 2)  # one CTA per instance: barriers are cheap, fewer V-cycles win (measured)
        solvers.append(sv)
    b = cdi.Batch(solvers)
    dts = np.array([w.dt for w in wls])
    best, tail, tune_ms = b.autotune(dts, 1)
    b.step(dts, 2)
    kb = max(2, min(steps, 5))
    ms_b = _timed_steps(lambda: b.step(dts, 1), kb, flush)
    loop_ms = _timed_steps(lambda: [sv.step(w.dt, 1) for sv, w in zip(solvers, wls)], 1, flush)
    cyc = [b.stats(i)["total_cycles"] for i in range(len(wls))]
    out["batched_sweep_512_fp32"] = {
        "value": cells * kb / (ms_b / 1e3) / 1e6, "unit": UNIT, "instances": len(wls), "cells": cells,
        "ms_per_step": ms_b / kb, "looped_single_grid_value": cells / (loop_ms / 1e3) / 1e6,
        "speedup_vs_looped": (loop_ms) / (ms_b / kb), "autotuned_threads": best, "autotuned_tail_bytes": tail,
        "autotune_ms_budget_by_threads": [[float(x) for x in row] for row in tune_ms],
        "mean_vcycles_per_step": float(np.mean(cyc)),
        "pressure_tol": PRESSURE_TOL}
    del b, solvers
    torch.cuda.empty_cache()
    # 3D drop 256^3, FP32-mixed (every field is 67 MB; the L2 is flushed before each step)
    wl = inputs.drop_3d(256)
    s = cdi.from_workload(wl, precision=cdi.FP32_MIXED, tol=PRESSURE_TOL)
    s.set_exec(cdi.EXEC_KERNELS)
    s.set_solver(PRESSURE_TOL, 100, cdi.WARM_PREV)  # extrapolation costs cycles on this transient (24 vs 21)
    s.set_smoothing(*SMOOTHING_3D)
    s.set_coarse_smoothing(*COARSE_SMOOTHING_3D)
    s.step(wl.dt, 5)
    k3 = 10
    cyc3 = []

    def one3():
        s.step(wl.dt, 1)
        cyc3.append(s.last_stats()["total_cycles_call"])
    ms3 = _timed_steps(one3, k3, flush)
    nbytes = sum(step_bytes(3, wl.cells, 4, c, sum(SMOOTHING_3D)) for c in cyc3)
    ach = nbytes / (ms3 / 1e3) / 1e9
    out["fp32_mixed_drop3d_256"] = {"value": wl.cells * k3 / (ms3 / 1e3) / 1e6, "unit": UNIT,
                                    "ms_per_step": ms3 / k3, "vcycles_per_step": float(np.mean(cyc3)),
                                    "pressure_tol": PRESSURE_TOL,
                                    "roofline": {"bound": "hbm", "kernel": "step", "achieved": ach, "peak": hbm,
                                                 "unit": "GB/s", "frac": ach / hbm, "peak_source": peak_kind,
                                                 "algorithmic_bytes_per_step": nbytes / k3}}
    del s
    torch.cuda.empty_cache()
    out["unet_warm_start_drop3d_64"] = unet_form(flush)
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        gpu_arm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
