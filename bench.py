"""Benchmark: sample-DoF-steps/s of the GPU implicit-Euler / Parareal path.

Linear solver (--solver): "banded" (default; band Cholesky factored once per
sample and step size, two substitutions per step) or "pcg" (batched
Jacobi-PCG).  Both pass the same oracle parity tests.

Default workload (the configuration the metric is quoted on that fits one
GPU): Parareal on one nominal sample of the 20k-node annulus in FP64 -- fine
dt = period/512 over 8 periods (4096 steps), coarse dt = 64 fine, 64 slices,
relative jump tolerance 1e-8, joule-loss QoI.  One bench step is one full
pass of the path on that input: per-sample value expansion, the Parareal
iterations (fine batches + coarse sweeps with the fused correction), the QoI
and the MLMC moment update, read back to device memory.  Throughput counts
serial-equivalent fine steps: 4096 x 19584 sample-DoF-steps per solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--precision fp64|mixed] [--solver banded|pcg]
                    [--workload parareal20k|parareal20k_short|mlmc20k|mlmc20k_short|mcsquare]

With N > 1 (torchrun) every rank runs an independent replica ("replicas
only": the Parareal solve of one sample has no cross-GPU exchange); value is
the units of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# before CUDA initialises: hardware queues for the pipelined Parareal streams
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------ workloads
def workload(name):
    from workloads import configs, meshes, params
    if name == "parareal20k":
        c = configs.PARAREAL_ANNULUS
        return dict(name="parareal_annulus20k", mesh=meshes.annulus("20k"),
                    params=params.annulus_nominal(1), t_end=c.periods * configs.PERIOD,
                    dt=c.dt, n_steps=c.n_steps, n_slices=c.n_slices, cf=c.coarse_factor,
                    par_tol=c.tol, qoi=c.qoi, cg_tol=1e-12)
    if name == "parareal20k_short":
        # profiling case: the same mesh, lanes and launch shapes as parareal20k
        # but 4 fine steps per slice (coarse step = 4 fine steps), so that one
        # launch of each kernel ends in well under a second
        c = configs.PARAREAL_ANNULUS
        return dict(name="parareal_annulus20k_short", mesh=meshes.annulus("20k"),
                    params=params.annulus_nominal(1), t_end=256 * c.dt, dt=c.dt, n_steps=256,
                    n_slices=c.n_slices, cf=4, par_tol=c.tol, qoi=c.qoi, cg_tol=1e-12)
    if name == "mlmc20k":
        c = configs.MLMC_ANNULUS
        return dict(name="mlmc_annulus20k", mesh=meshes.annulus("20k"), mlmc=c,
                    params=[params.annulus_samples(n, l) for l, n in enumerate(c.n_per_level)],
                    t_end=c.periods * configs.PERIOD, qoi=c.qoi, cg_tol=1e-12,
                    n_steps=None, dt=configs.level_dt(0), n_slices=1, cf=1, par_tol=0.0)
    if name == "mlmc20k_short":
        # profiling case: the MLMC workload's mesh, inputs and launch shapes over
        # one period with 608/152/38/16 samples (level 0 fills 4 CTAs per SM)
        c = configs.MLMCAnnulus(periods=1, n_per_level=(608, 152, 38, 16))
        return dict(name="mlmc_annulus20k_short", mesh=meshes.annulus("20k"), mlmc=c,
                    params=[params.annulus_samples(n, l) for l, n in enumerate(c.n_per_level)],
                    t_end=c.periods * configs.PERIOD, qoi=c.qoi, cg_tol=1e-12,
                    n_steps=None, dt=configs.level_dt(0), n_slices=1, cf=1, par_tol=0.0)
    if name == "mcsquare":
        c = configs.MC_SQUARE
        return dict(name="mc_square16", mesh=meshes.unit_square(16),
                    params=params.square_samples(c.n_samples), t_end=c.t_end,
                    dt=c.t_end / c.n_steps, n_steps=c.n_steps, n_slices=1, cf=1, par_tol=0.0,
                    qoi=c.qoi, cg_tol=1e-13)
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                s, m = float(f[0]), float(f[1])
            except Exception:
                continue
            sm.append(s)
            mx = m
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm if mx and s > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ bytes model
def algorithmic_bytes(n_free, nnz, lane_iters, lane_steps, lanes_per_value, precision):
    """Algorithmic DRAM bytes of the stepping kernel (per launch set).

    Per lane and CG iteration, each row moves its matrix row (z/n values plus
    the inverse diagonal, shared by `lanes_per_value` lanes) and 12 lane-vector
    words: SpMV reads p, writes q; the update reads x, p, r, q and writes
    x, r, z; the direction update reads z, p and writes p.  Per lane and
    step, the right-hand side and the QoI add two matrix rows and 10 words.
    Mixed precision: FP32 values and FP32 p/q copies in the SpMV.
    """
    zn = nnz / n_free
    wv = 4 if precision == "mixed" else 8
    per_it = (wv * zn + 8) / lanes_per_value + 12 * 8
    if precision == "mixed":
        per_it += 2 * 4 - 8  # p32 written, q32 in place of q; SpMV reads p32
    per_step = 2 * 8 * zn / lanes_per_value + 10 * 8
    return n_free * (lane_iters * per_it + lane_steps * per_step)


def algorithmic_flops(n_free, nnz, lane_iters, lane_steps):
    """Algorithmic FP64 flops of the Jacobi-PCG stepping (per launch set).

    Per lane, row and CG iteration: the SpMV row (2 z/n), three dot products
    (p.q, r.z, r.r: 6), three axpys (x, r, p: 6) and z = D^-1 r (1).  Per
    lane, row and step: the residual b - A a0 (2 z/n + 4), the source sum
    and the QoI with y = M a (2 z/n + 4).
    """
    zn = nnz / n_free
    return n_free * (lane_iters * (2 * zn + 13) + lane_steps * (4 * zn + 8))


def banded_flops(n_free, nnz, bw, lane_steps):
    """Algorithmic FP64 flops of banded-solver stepping: per lane-step the
    forward and backward substitutions (sum over rows of min(i, bw) FMAs each,
    ~ n bw - bw^2/2) plus the right-hand side and the QoI / y = M a SpMV."""
    subst = 2 * 2 * (n_free * bw - bw * bw / 2.0)
    return lane_steps * (subst + n_free * (2.0 * nnz / n_free + 10.0))


# FP64 peak from the unit counts (fallback when the in-tree measurement is
# unavailable): 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------------ oracle on the host cores
# The oracle is plain FP64 numpy/scipy.  A spawn pool of one process per host
# core runs its independent pieces: the fine propagations of one Parareal
# iteration (the slices, as the method distributes them over cores) and the
# level pairs of MLMC samples.  Each worker builds its propagators once.
_W = {}


def _mesh_of(name):
    from workloads import meshes
    if name not in _W.setdefault("meshes", {}):
        _W["meshes"][name] = (meshes.unit_square(16) if name == "square16"
                              else meshes.annulus(name.replace("annulus", "")))
    return _W["meshes"][name]


def _init_fine(mesh_name, prow, dt, steps_per_slice, qoi):
    from oracle import fem, stepper
    d = fem.Discretisation(_mesh_of(mesh_name), prow)
    _W["fine"] = (stepper.ImplicitEuler(d, dt), steps_per_slice, qoi)


def _fine_task(task):
    s, u = task
    prop, S, qoi = _W["fine"]
    a, raw, _ = prop.run(u, S, k0=s * S, qoi=qoi)
    return a, raw


def _pair_task(task):
    """(Q_l, Q_{l-1}) of one sample from a(0) = 0 over `periods` periods."""
    from oracle import mlmc
    from workloads import configs
    mesh_name, prow, level, periods, qoi = task
    return mlmc.level_pair(_mesh_of(mesh_name), prow, level, configs.level_dt,
                           lambda k: configs.level_steps(periods, k), qoi)


def _serial_task(task):
    """Serial implicit Euler of one sample for n_steps (MC workload)."""
    from oracle import stepper
    mesh_name, prow, dt, n_steps, qoi = task
    q, _, _ = stepper.solve_sample(_mesh_of(mesh_name), prow, dt, n_steps, qoi)
    return q


def _init_worker(ready, init, initargs):
    if init is not None:
        init(*initargs)
    with ready.get_lock():
        ready.value += 1


class OraclePool:
    """One spawn process per host core; returns once every worker has run its
    initializer (so that set-up is not timed)."""

    def __init__(self, init=None, initargs=()):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = os.cpu_count() or 1
        # one process per core, each single-threaded (the children read these
        # when they import numpy)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        ready = ctx.Value("i", 0)
        self.pool = ctx.Pool(processes=self.cores, initializer=_init_worker,
                             initargs=(ready, init, initargs))
        t0 = time.time()
        while ready.value < self.cores and time.time() - t0 < 600:
            time.sleep(0.05)

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_parareal_pool(wl):
    S = wl["n_steps"] // wl["n_slices"]
    return OraclePool(_init_fine, (wl["mesh"].name, wl["params"][0], wl["dt"], S, wl["qoi"]))


def oracle_parareal(wl, pool):
    """The oracle's Parareal on the workload's sample with the fine slices of
    each iteration on the pool's processes; returns (seconds, result).  The
    workers' fine factorisations were built with the pool; the main process
    builds its discretisation and the coarse factor inside the timed solve."""
    from oracle import fem, parareal

    def fmap(slices, starts):
        return pool.pool.map(_fine_task, list(zip(slices, starts)))

    t0 = time.perf_counter()
    d = fem.Discretisation(wl["mesh"], wl["params"][0])
    ref = parareal.parareal_sample(d, wl["dt"], wl["n_steps"], wl["n_slices"], wl["cf"],
                                   wl["par_tol"], wl["qoi"], fine_map=fmap)
    return time.perf_counter() - t0, ref


def oracle_pairs(tasks, pool):
    """Level pairs of MLMC samples on the pool: (seconds, results)."""
    t0 = time.perf_counter()
    out = pool.pool.map(_pair_task, tasks, chunksize=1)
    return time.perf_counter() - t0, out


def static_config(wl, args, n_free, nnz, world=1):
    """The workload part of the JSON line's config, the same in both arms."""
    if "mlmc" in wl:
        c = wl["mlmc"]
        return {"workload": wl["name"], "n_free": n_free, "levels": len(c.n_per_level),
                "n_per_level": list(c.n_per_level), "periods": c.periods,
                "solver": args.solver, "precision": args.precision,
                "solve_steps": c.solve_steps(), "parallelism": f"replicas x{world}"}
    return {"workload": wl["name"], "mesh": wl["mesh"].name, "n_free": n_free, "nnz": nnz,
            "samples": int(wl["params"].shape[0]), "steps": wl["n_steps"], "dt": wl["dt"],
            "slices": wl["n_slices"], "coarse_factor": wl["cf"], "parareal_tol": wl["par_tol"],
            "precision": args.precision, "solver": args.solver,
            "parallelism": f"replicas x{world}"}


def mesh_pattern(mesh):
    """Free unknowns and nonzeros of the P1 pattern over them (topology only)."""
    free = [v for v in range(len(mesh.xy)) if not mesh.dirichlet[v]]
    fid = {v: k for k, v in enumerate(free)}
    pairs = set()
    for t in mesh.tri:
        ids = [fid.get(int(v)) for v in t]
        for a in ids:
            for b in ids:
                if a is not None and b is not None:
                    pairs.add((a, b))
    return len(free), len(pairs)


def mlmc_subset(c, n_each=2):
    """Per-level sample subset of the MLMC workload: the first n_each samples
    of every level (the level-pair QoIs the GPU run is checked against)."""
    return [(l, j) for l in range(c.n_levels) for j in range(min(n_each, c.n_per_level[l]))]


def run_reference(args, wl, rank, world):
    """The oracle on the host cores, timed on the same workload as the GPU arm."""
    if rank != 0:
        return
    n_free, nnz = mesh_pattern(wl["mesh"])
    vals, secs = [], []
    if "mlmc" in wl:
        c = wl["mlmc"]
        sub = mlmc_subset(c)
        units = sum((c.steps(l) + (c.steps(l - 1) if l else 0)) for l, _ in sub) * n_free
        what = (f"level pairs of {len(sub)} samples (the first 2 of each level) of the MLMC "
                f"workload, serial implicit Euler with banded Cholesky per sample")
        pool = OraclePool()
        tasks = [(wl["mesh"].name, wl["params"][l][j], l, c.periods, c.qoi) for l, j in sub]
        run = lambda: oracle_pairs(tasks, pool)[0]
    elif wl["n_slices"] > 1:
        units = wl["n_steps"] * n_free
        what = (f"the oracle's Parareal of the workload ({wl['n_slices']} slices, tolerance "
                f"{wl['par_tol']:g}): the fine slices of each iteration on the pool's "
                f"processes, the coarse sweep and the Eq. 12 correction in the main process")
        pool = oracle_parareal_pool(wl)
        run = lambda: oracle_parareal(wl, pool)[0]
    else:
        units = wl["n_steps"] * n_free * wl["params"].shape[0]
        what = "every sample of the workload, serial implicit Euler with banded Cholesky"
        pool = OraclePool()
        tasks = [(wl["mesh"].name, row, wl["dt"], wl["n_steps"], wl["qoi"]) for row in wl["params"]]

        def run():
            t0 = time.perf_counter()
            pool.pool.map(_serial_task, tasks)
            return time.perf_counter() - t0
    try:
        for i in range(args.warmup + args.steps):
            t = run()
            if i >= args.warmup:
                vals.append(units / t)
                secs.append(t)
    finally:
        pool.close()
    cores = pool.cores
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": "sample-DoF-steps/s", "value": value,
            "unit": "sample-DoF-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": static_config(wl, args, n_free, nnz, world),
            "e2e": {"value": value, "unit": "sample-DoF-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": "sample-DoF-steps/s", "cores": cores,
                             "kind": "oracle", "sample": what + f"; {cores} host cores"}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, wl, rank, world, dist):
    import numpy as np
    import torch

    from paper_2507_19246_gb300 import mqs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    prec = mqs.MQS_MIXED if args.precision == "mixed" else mqs.MQS_FP64
    ctx = mqs.Context(dev, stream.cuda_stream)
    mesh_id = ctx.upload_mesh(wl["mesh"])
    n_free, nnz = ctx.mesh_info(mesh_id)
    p_host = torch.from_numpy(wl["params"]).pin_memory()
    p_dev = p_host.to(f"cuda:{dev}")
    ns = p_host.shape[0]
    q_dev = torch.zeros((ns, 2), dtype=torch.float64, device=f"cuda:{dev}")
    # linear-solve stopping: FP64 PCG to the parity tolerance; mixed forms to
    # 1e-10 (QoI within 1e-6 of the FP64 oracle); the banded mixed form caps
    # its FP64 refinement sweeps, the PCG forms their iterations
    mixed = args.precision == "mixed"
    tol_lin = 1e-10 if mixed else wl["cg_tol"]
    max_lin = (12 if mixed else 1) if args.solver == "banded" else 20000
    q_host = torch.zeros((ns, 2), dtype=torch.float64).pin_memory()
    flush = torch.empty(int(512e6) // 4, dtype=torch.float32, device=f"cuda:{dev}")
    # measured FP64 / FP32 peaks of this GPU (in-tree FMA-chain microbenchmark)
    peak64 = mqs.mqs_measure_peak(dev, stream.cuda_stream, mqs.MQS_FP64)
    peak32 = mqs.mqs_measure_peak(dev, stream.cuda_stream, mqs.MQS_MIXED)

    def one_step(params_src, qoi_dst, n_slices=None):
        b = mqs.mqs_set_samples(ctx.h, mesh_id, params_src)
        if args.solver == "banded":
            mqs.mqs_set_solver(ctx.h, b, mqs.MQS_SOLVER_BANDED)
        mqs.mqs_set_time(ctx.h, b, 0.0, wl["t_end"], 50.0, wl["qoi"])
        m = wl["n_slices"] if n_slices is None else n_slices
        k = mqs.mqs_propagate(ctx.h, b, 0, wl["dt"], 0.0, m, wl["cf"] if m > 1 else 1,
                              m, wl["par_tol"], prec, tol_lin, max_lin)
        mqs.mqs_mlmc_accumulate(ctx.h, b, 0)
        mqs.mqs_read_qoi(ctx.h, b, qoi_dst)
        st = mqs.mqs_read_stats(ctx.h, b)
        mqs.mqs_free_batch(ctx.h, b)
        return k, st

    mqs.mqs_mlmc_reset(ctx.h, 1)
    for _ in range(args.warmup):
        one_step(p_dev, q_dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # ---- device-resident timed region
    times, ks, stats = [], [], []
    launches0 = ctx.profile_read()[0]
    ctx.profile(True)
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)                       # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            k, st = one_step(p_dev, q_dev)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            ks.append(k)
            stats.append(st)
    prof = ctx.profile_read()
    ctx.profile(False)
    launches = int(prof[0] - launches0)
    torch.cuda.synchronize()
    # ---- end-to-end through the public API from pinned host memory
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step(p_host, q_host.numpy())
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    q = q_dev.cpu().numpy()
    # ---- max over ranks
    ms_total = sum(times)
    if dist:
        t = torch.tensor([ms_total, sum(e2e_times)], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total, e2e_total = t.tolist()
    else:
        e2e_total = sum(e2e_times)
    units = float(ns) * wl["n_steps"] * n_free           # serial-equivalent sample-DoF-steps
    value = world * units * args.steps / (ms_total / 1e3)
    e2e_value = world * units * len(e2e_times) / (e2e_total / 1e3)
    if rank != 0:
        ctx.close()
        return
    st = stats[-1]
    # ---- roofline of the dominant kernel from the live CUDA-event timings of
    # the timed region: the stepping kernel (Parareal fine chunks, several in
    # flight on their own streams) against the time at least one of them ran
    step_ms, step_n, sweep_ms, sweep_n = prof[2], prof[1], prof[4], prof[3]
    step_cov, sweep_cov = prof[5], prof[6]
    bw = mqs.mqs_mesh_bandwidth(ctx.h, mesh_id) if args.solver == "banded" else 0
    if args.solver == "banded":
        step_flops = sum(banded_flops(n_free, nnz, bw, s[6]) for s in stats)
        sweep_flops = sum(banded_flops(n_free, nnz, bw, s[7]) for s in stats)
    else:
        step_flops = sum(algorithmic_flops(n_free, nnz, s[4], s[6]) for s in stats)
        sweep_flops = sum(algorithmic_flops(n_free, nnz, s[5], s[7]) for s in stats)
    lpv = 32 if wl["n_slices"] % 32 == 0 else wl["n_slices"]
    step_bytes = sum(algorithmic_bytes(n_free, nnz, s[4], s[6], lpv, args.precision)
                     for s in stats)
    peaks, _ = _peaks()
    peak_fp = peak64 if args.precision == "fp64" else peak32
    dominant = "stepping" if step_cov >= sweep_cov else "coarse_sweep"
    d_flops, d_cov = (step_flops, step_cov) if dominant == "stepping" else (sweep_flops, sweep_cov)
    achieved = d_flops / (d_cov / 1e3) / 1e12 if d_cov > 0 else 0.0
    # DRAM traffic per launch from a recorded single-pass ncu capture of the
    # same kernel source (null once that source file has changed)
    traffic = None
    try:
        import hashlib
        key = f"{wl['name']}:{args.precision}:{args.solver}:{dominant}"
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(key)
        if tr:
            src = os.path.join(ROOT, "paper_2507_19246_gb300", "csrc", tr["source_file"])
            cur = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            if tr.get("source_sha256_16") == cur:
                traffic = tr["bytes_per_launch"]
    except Exception:
        traffic = None
    clocks = clk.summary()
    line = {
        "metric": "sample-DoF-steps/s", "value": value, "unit": "sample-DoF-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": static_config(wl, args, n_free, nnz, world),
        "l2": "flushed (512 MB write) before every timed step",
        "linear_tol": tol_lin, "parareal_iters": ks[-1], "bandwidth": bw,
        "p50_ms": statistics.median(times),
        "p99_ms": sorted(times)[min(len(times) - 1, int(0.99 * len(times)))],
        "time_to_solution_s": ms_total / args.steps / 1e3,
        "effort_solve_steps": st[1], "serial_equivalent_solve_steps": st[2],
        "qoi": float(q[0, 0]),
        "e2e": {"value": e2e_value, "unit": "sample-DoF-steps/s",
                "h2d_bytes_per_step": int(p_host.numel() * 8), "d2h_bytes_per_step": int(ns * 2 * 8)},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak_fp,
                     "unit": "TFLOP/s", "frac": achieved / peak_fp if peak_fp else None,
                     "traffic": traffic,
                     "peak_source": ("measured in-tree: FP64 FMA chains on every SM "
                                     "(mqs_measure_peak), " if args.precision == "fp64" else
                                     "measured in-tree: FP32 FMA chains (mqs_measure_peak), ")
                                    + f"unit-count figure {FP64_PEAK_DERIVED:.3f} TFLOP/s FP64",
                     "achieved_over": "time during which at least one launch of the kernel ran",
                     "kernel_ms_per_step": {
                         "stepping_sum": step_ms / args.steps, "stepping_covered": step_cov / args.steps,
                         "coarse_sweep_sum": sweep_ms / args.steps,
                         "coarse_sweep_covered": sweep_cov / args.steps},
                     "coarse_sweep_tflops": sweep_flops / (sweep_cov / 1e3) / 1e12 if sweep_cov else 0.0,
                     "algorithmic_dram_gbs": step_bytes / (step_cov / 1e3) / 1e9 if step_cov else 0.0,
                     "hbm_peak_gbs": peaks.get("hbm_gbs")},
        "peaks_measured": {"fp64_tflops": peak64, "fp32_tflops": peak32},
        "clocks": clocks,
    }
    # ---- the paper's Parareal speedup s (Sec. II-C): the GPU's own serial fine
    # solve of the same sample against the Parareal solve
    if wl["n_slices"] > 1 and not args.no_extras:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(p_dev, q_dev, n_slices=1)
        e1.record(stream)
        e1.synchronize()
        serial_ms = e0.elapsed_time(e1)
        line["gpu_serial_fine_ms"] = serial_ms
        line["parareal_speedup_vs_gpu_serial"] = serial_ms / statistics.median(times)
    # ---- MLMC time-to-RMSE (configs' MLMC workload), FP64 and mixed
    if not args.no_extras and wl["name"] == "parareal_annulus20k":
        line["mlmc"] = mlmc_records(args, ctx, mqs, torch, stream)
    # ---- the request server under a Poisson stream (p50/p99 latency)
    if not args.no_extras and wl["name"] == "parareal_annulus20k":
        line["serving"] = serving_record(ctx, mqs)
    # ---- CPU baseline: the oracle on the host cores (after the GPU work)
    if not args.no_cpu_baseline and wl["n_slices"] > 1:
        pool = oracle_parareal_pool(wl)
        try:
            secs, ref = oracle_parareal(wl, pool)
        finally:
            pool.close()
        line["cpu_baseline"] = {
            "value": units / secs, "unit": "sample-DoF-steps/s", "cores": pool.cores,
            "kind": "oracle",
            "sample": (f"one Parareal solve of the workload by the oracle ({ref['iters']} "
                       f"iterations, {secs:.1f} s): fine slices of each iteration on "
                       f"{pool.cores} host processes, coarse sweep and correction in the main "
                       f"process")}
    print(json.dumps(line), flush=True)
    ctx.close()


def mlmc_records(args, ctx, mqs, torch, stream):
    """MLMC estimate (Eq. 9) of the configs' MLMC workload on the 20k annulus
    (4 levels, N_l = 4096/1024/256/64, 4 periods) in FP64 and in mixed
    precision: time-to-RMSE (one timed estimate each after a one-level
    warm-up), throughput, and the QoI error of the level pairs of a per-level
    sample subset against the FP64 oracle."""
    import numpy as np

    from workloads import configs
    wl = workload("mlmc20k")
    c = wl["mlmc"]
    mesh_id = ctx.upload_mesh(wl["mesh"])
    n_free, _ = ctx.mesh_info(mesh_id)
    p_dev = [torch.from_numpy(p).cuda() for p in wl["params"]]
    sub = mlmc_subset(c)
    chunk = 1024
    out = {"workload": wl["name"], "n_per_level": list(c.n_per_level), "periods": c.periods,
           "repeats": 1, "subset": "first 2 samples of every level"}

    def estimate(prec, tol, sweeps, levels=None):
        mqs.mqs_mlmc_reset(ctx.h, c.n_levels)
        qsub = {}
        for l, N in enumerate(c.n_per_level):
            if levels is not None and l not in levels:
                continue
            for s0 in range(0, N, chunk):
                b = mqs.mqs_set_samples(ctx.h, mesh_id, p_dev[l][s0:s0 + chunk])
                mqs.mqs_set_solver(ctx.h, b, mqs.MQS_SOLVER_BANDED)
                mqs.mqs_set_time(ctx.h, b, 0.0, wl["t_end"], 50.0, wl["qoi"])
                mqs.mqs_propagate(ctx.h, b, l, configs.level_dt(l),
                                  configs.level_dt(l - 1) if l else 0.0, 1, 1, 1, 0.0, prec,
                                  tol, sweeps)
                mqs.mqs_mlmc_accumulate(ctx.h, b, l)
                if s0 == 0:
                    qd = torch.empty((min(N, chunk), 2), dtype=torch.float64, device="cuda")
                    mqs.mqs_read_qoi(ctx.h, b, qd)
                    qsub[l] = qd
                mqs.mqs_free_batch(ctx.h, b)
        return mqs.mqs_mlmc_readout(ctx.h, c.n_levels), qsub

    runs = {}
    # mixed: FP32 factor, FP64 residuals; a relative residual of 2e-6 is met
    # after two FP32 solves per step on this mesh (one refinement), which keeps
    # the QoI within ~1e-9 of FP64 -- far inside the 1e-6 bound
    for name, prec, tol, sweeps in (("fp64", mqs.MQS_FP64, 1e-12, 1),
                                    ("mixed", mqs.MQS_MIXED, 2e-6, 4)):
        estimate(prec, tol, sweeps, levels=[c.n_levels - 1])      # warm-up: the finest level
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            e0.record(stream)
            (lv, est, rmse), qsub = estimate(prec, tol, sweeps)
            e1.record(stream)
            e1.synchronize()
            wall = time.perf_counter() - t0
        qs = {l: qsub[l].cpu().numpy() for l in qsub}
        runs[name] = qs
        out[name] = {"time_to_rmse_s": wall, "device_s": e0.elapsed_time(e1) / 1e3,
                     "estimate": est, "rmse": rmse, "levels": lv.tolist(),
                     "sample_dof_steps_per_s": c.solve_steps() * n_free / wall,
                     "linear_tol": tol, "max_sweeps": sweeps, "clocks": clk.summary()}
    # the oracle's level pairs of the subset, on the host cores
    pool = OraclePool()
    try:
        secs, ref = oracle_pairs([(wl["mesh"].name, wl["params"][l][j], l, c.periods, c.qoi)
                                  for l, j in sub], pool)
    finally:
        pool.close()
    cores = pool.cores
    for name in ("fp64", "mixed"):
        errs = []
        for (l, j), (qf, qc) in zip(sub, ref):
            errs.append(abs(runs[name][l][j, 0] - qf) / abs(qf))
            if l:
                errs.append(abs(runs[name][l][j, 1] - qc) / abs(qc))
        out[name]["qoi_max_rel_err_vs_oracle"] = float(max(errs))
    out["oracle_subset_s"] = secs
    out["oracle_cores"] = cores
    out["mixed_over_fp64_throughput"] = (out["mixed"]["sample_dof_steps_per_s"] /
                                         out["fp64"]["sample_dof_steps_per_s"])
    return out


def serving_record(ctx, mqs, n_requests=240, rate=40.0, seed=20250725, n_streams=32):
    """The request server under a Poisson stream (the configs' serving
    workload, scaled so that the run takes seconds): level samples (levels
    0-2 with their level-(l-1) companions) and Parareal slices, on the 5k,
    20k and 80k annuli with 256 or 1024 steps, submitted at their arrival
    times; per-request latency from submission to completion."""
    import numpy as np

    from workloads import configs, meshes, params
    rng = np.random.default_rng(seed)
    names = ["5k", "20k", "80k"]
    mids = {nm: ctx.upload_mesh(meshes.annulus(nm)) for nm in names}
    nfree = {nm: ctx.mesh_info(mids[nm])[0] for nm in names}
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    reqs = []
    for j in range(n_requests):
        nm = rng.choice(names, p=[0.5, 0.4, 0.1])
        steps = int(rng.choice([256, 1024]))
        prow = params.annulus_samples(1, 3, seed=seed, first=j)[0]
        if rng.random() < 0.7:
            l = int(rng.integers(0, 3))
            lanes = [(configs.level_dt(l), steps)]
            if l:
                lanes.append((configs.level_dt(l - 1), steps // 2))
            reqs.append((nm, prow, mqs.MQS_REQ_LEVEL, lanes, 0))
        else:
            k0 = int(rng.integers(0, 4)) * steps
            reqs.append((nm, prow, mqs.MQS_REQ_SLICE, [(configs.level_dt(2), steps)], k0))
    units = sum(nfree[r[0]] * sum(n for _, n in r[3]) for r in reqs)
    lat, done = [], {}
    with mqs.Server(ctx, n_streams=n_streams, max_batch_lanes=608) as srv:
        t0 = time.perf_counter()
        nxt, peak_inflight, peak_queue = 0, 0, 0
        ids = {}
        while len(done) < n_requests:
            now = time.perf_counter() - t0
            while nxt < n_requests and arrivals[nxt] <= now:
                nm, prow, kind, lanes, k0 = reqs[nxt]
                (dt, n), prev = lanes[0], (lanes[1] if len(lanes) > 1 else (0.0, 0))
                rid = srv.submit(mids[nm], prow, kind, mqs.MQS_QOI_JOULE, 0.0, dt, n,
                                 dt_prev=prev[0], n_steps_prev=prev[1], k0=k0)
                ids[rid] = nxt
                nxt += 1
            inf, q = srv.progress()
            peak_inflight, peak_queue = max(peak_inflight, inf), max(peak_queue, q)
            for rid, qq, st, tm in zip(*srv.poll()):
                done[int(rid)] = (tm[2] - tm[0], tm[1] - tm[0], int(st), tm[2])
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
    lat = np.array([v[0] for v in done.values()])
    wait = np.array([v[1] for v in done.values()])
    last_done = max(v[3] for v in done.values())
    return {"requests": n_requests, "rate_per_s": rate, "streams": n_streams,
            "mix": "70% level samples (levels 0-2, companions for l > 0), 30% Parareal slices; "
                   "meshes 5k/20k/80k with p = 0.5/0.4/0.1; 256 or 1024 steps",
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "queue_wait_p50_s": float(np.percentile(wait, 50)),
            "queue_wait_p99_s": float(np.percentile(wait, 99)),
            "sample_dof_steps_per_s": units / last_done, "wall_s": wall,
            "peak_in_flight": peak_inflight, "peak_queued": peak_queue,
            "failed": int(sum(1 for v in done.values() if v[2]))}


def run_mlmc_parareal_80k(args):
    """MLMC with Parareal on the finest level (Sec. II-D) on the 80k annulus:
    5 levels, dt_l = period/(64 2^l) over 8 periods, level 4 by Parareal with
    32 slices and coarse propagator = level 2, its level-3 companion solve
    beside it.  Sample counts are the configuration's N_l = 8192/2048/512/128/32
    times --scale (the full counts are ~1e15 FP64 FMAs, about 30 minutes at
    the GPU's FP64 peak).  One estimate per step; QoIs of the first sample of
    levels 0 and 1 against the oracle."""
    import numpy as np
    import torch

    from paper_2507_19246_gb300 import mqs, planner
    from workloads import configs, meshes, params
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = mqs.Context(0, stream.cuda_stream)
    mesh = meshes.annulus("80k")
    mid = ctx.upload_mesh(mesh)
    n_free, _ = ctx.mesh_info(mid)
    periods, L, M, cf, tol = 8, 5, 32, 4, 1e-8
    N = [max(2, int(round(n * args.scale))) for n in (8192, 2048, 512, 128, 32)]
    T = periods * configs.PERIOD
    dts = [configs.level_dt(l) for l in range(L)]
    steps = [configs.level_steps(periods, l) for l in range(L)]
    prm = [params.annulus_samples(N[l], l, seed=20250725 + 7) for l in range(L)]
    p_dev = [torch.from_numpy(p).cuda() for p in prm]
    chunk = 128
    info = {}

    def estimate():
        mqs.mqs_mlmc_reset(ctx.h, L)
        per_level, ks, q0 = [], [], {}
        for l in range(L):
            t0 = time.perf_counter()
            for s0 in range(0, N[l], chunk):
                b = mqs.mqs_set_samples(ctx.h, mid, p_dev[l][s0:s0 + chunk])
                mqs.mqs_set_solver(ctx.h, b, mqs.MQS_SOLVER_BANDED)
                mqs.mqs_set_time(ctx.h, b, 0.0, T, 50.0, configs.QOI_JOULE)
                slices = M if l == L - 1 else 1
                k = mqs.mqs_propagate(ctx.h, b, l, dts[l], dts[l - 1] if l else 0.0, slices,
                                      cf if slices > 1 else 1, slices, tol, mqs.MQS_FP64,
                                      1e-12, 1)
                if slices > 1:
                    ks.append(k)
                mqs.mqs_mlmc_accumulate(ctx.h, b, l)
                if s0 == 0 and l < 2:
                    qd = torch.empty((min(chunk, N[l]), 2), dtype=torch.float64, device="cuda")
                    mqs.mqs_read_qoi(ctx.h, b, qd)
                    q0[l] = qd[0].cpu().numpy()
                mqs.mqs_free_batch(ctx.h, b)
            torch.cuda.synchronize()
            per_level.append(time.perf_counter() - t0)
        return mqs.mqs_mlmc_readout(ctx.h, L), per_level, ks, q0

    for _ in range(args.warmup):
        estimate()
    times, res = [], None
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            res = estimate()
            times.append(time.perf_counter() - t0)
    (lv, est, rmse), per_level, ks, q0 = res
    slots = ctx.lane_slots()
    n_para, m_plan = planner.plan_finest_level(N[-1], steps[-1], steps[-2], slots, steps[-1], cf)
    units = sum(N[l] * (steps[l] + (steps[l - 1] if l else 0)) for l in range(L)) * n_free
    pool = OraclePool()
    try:
        secs, ref = oracle_pairs([("annulus80k", prm[l][0], l, periods, configs.QOI_JOULE)
                                  for l in range(2)], pool)
    finally:
        pool.close()
    errs = []
    for l, (qf, qc) in enumerate(ref):
        errs.append(abs(q0[l][0] - qf) / abs(qf))
        if l:
            errs.append(abs(q0[l][1] - qc) / abs(qc))
    line = {"metric": "sample-DoF-steps/s", "value": units * len(times) / sum(times),
            "unit": "sample-DoF-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "mlmc_parareal_annulus80k", "n_free": n_free, "levels": L,
                       "n_per_level": N, "scale_of_configured_counts": args.scale,
                       "periods": periods, "parareal_level": L - 1, "slices": M,
                       "coarse_level": L - 3, "parareal_tol": tol, "solver": "banded",
                       "precision": "fp64", "parallelism": "replicas x1"},
            "time_to_rmse_s": statistics.median(times), "estimate": est, "rmse": rmse,
            "levels": lv.tolist(), "level_seconds": per_level, "parareal_iters": ks,
            "planner": {"lane_slots": slots, "n_c_para_eq25": n_para, "slices_planned": m_plan},
            "qoi_max_rel_err_vs_oracle_levels_0_1": float(max(errs)),
            "oracle_seconds": secs, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_mlmc(args, wl):
    """One MLMC estimate (Eq. 9) per step: every level's samples, both solves
    of each level pair, moments, readout; time-to-RMSE from upload to readout."""
    import torch

    from paper_2507_19246_gb300 import mqs

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = mqs.Context(0, stream.cuda_stream)
    from workloads import configs
    c = wl["mlmc"]
    mesh_id = ctx.upload_mesh(wl["mesh"])
    n_free, nnz = ctx.mesh_info(mesh_id)
    prec = mqs.MQS_MIXED if args.precision == "mixed" else mqs.MQS_FP64
    p_dev = [torch.from_numpy(p).cuda() for p in wl["params"]]
    chunk = 1024
    L = c.n_levels

    def estimate():
        mqs.mqs_mlmc_reset(ctx.h, L)
        for l, N in enumerate(c.n_per_level):
            for s0 in range(0, N, chunk):
                b = mqs.mqs_set_samples(ctx.h, mesh_id, p_dev[l][s0:s0 + chunk])
                if args.solver == "banded":
                    mqs.mqs_set_solver(ctx.h, b, mqs.MQS_SOLVER_BANDED)
                mqs.mqs_set_time(ctx.h, b, 0.0, wl["t_end"], 50.0, wl["qoi"])
                mqs.mqs_propagate(ctx.h, b, l, configs.level_dt(l),
                                  configs.level_dt(l - 1) if l else 0.0, 1, 1, 1, 0.0, prec,
                                  1e-12 if prec == mqs.MQS_FP64 else 1e-10,
                                  (12 if prec == mqs.MQS_MIXED else 1) if args.solver == "banded"
                                  else 20000)
                mqs.mqs_mlmc_accumulate(ctx.h, b, l)
                mqs.mqs_free_batch(ctx.h, b)
        return mqs.mqs_mlmc_readout(ctx.h, L)

    for _ in range(args.warmup):
        estimate()
    torch.cuda.synchronize()
    times, res = [], None
    ctx.profile(True)
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            res = estimate()
            times.append(time.perf_counter() - t0)
    prof = ctx.profile_read()
    ctx.profile(False)
    lv, est, rmse = res
    units = c.solve_steps() * n_free
    line = {"metric": "sample-DoF-steps/s", "value": units * len(times) / sum(times),
            "unit": "sample-DoF-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
            "config": static_config(wl, args, n_free, None),
            "time_to_rmse_s": statistics.median(times), "estimate": est, "rmse": rmse,
            "levels": lv.tolist(), "clocks": clk.summary(),
            "kernel_ms": {"stepping": prof[2] / len(times), "coarse_sweep": prof[4] / len(times)}}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 1 for mlmcpar80k, whose step is a whole "
                    "MLMC estimate of several minutes)")
    ap.add_argument("--warmup", type=int, default=None,
                    help="untimed warm-up steps (default 3; 1 for mlmcpar80k)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="parareal20k",
                    choices=["parareal20k", "parareal20k_short", "mcsquare", "mlmc20k",
                             "mlmc20k_short", "mlmcpar80k"])
    ap.add_argument("--scale", type=float, default=1.0 / 16,
                    help="mlmcpar80k: fraction of the configured sample counts")
    ap.add_argument("--solver", default="banded", choices=["pcg", "banded"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the GPU serial solve and the MLMC FP64/mixed records")
    args = ap.parse_args()
    long_step = args.workload == "mlmcpar80k"
    if args.steps is None:
        args.steps = 1 if long_step else 5
    if args.warmup is None:
        args.warmup = 1 if long_step else 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.workload == "mlmcpar80k":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the MLMC+Parareal 80k "
                              "workload is measured on the GPU only (the oracle needs hours "
                              "for its level-4 samples)"}), flush=True)
            return
        run_mlmc_parareal_80k(args)
        return
    wl = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.workload.startswith("mlmc20k"):
        run_mlmc(args, wl)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, wl, rank, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
