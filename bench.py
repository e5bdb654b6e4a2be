"""Benchmark: W1 solves/s at 512x512 on the GB300 (one JSON line on stdout).

Workload (512x512 image-shaped pairs, 6-level cascade 16->512, both norms):
one step = a batch of B fresh density pairs (already resident in HBM) solved
with the L1 and with the L2 ground norm through w1_solve_batch, i.e. 2B full
Algorithm-3 solves, each batch ending with the read-back of its W1 values.
The L2 cache is flushed (a 256 MiB write) before every step, inside the timed
region.

Also measured in the same run:
  e2e      : the same solves through w1_solve_host (host densities, H2D copies
             and the D2H result inside the timed region);
  roofline : the streaming step kernel on an 8192x8192 grid (1.9 GB of state,
             far above L2), 28 algorithmic bytes per node and step, timed with
             CUDA events on the stream it is launched on;
  cpu_baseline: the FP64 oracle on this host's cores (one process per core,
             all at once; one_core_value: a single process alone), per-level
             step cost measured on a bounded sample and scaled by the oracle's
             own per-level iteration counts for the same pairs
             (oracle/iter_table.json).

--impl reference runs that oracle arm alone (CPU only).
Multi-GPU (torchrun): every rank solves its own pairs (independent replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Many concurrent solves use many streams; give the context 32 hardware work
# queues instead of the default 8 (must be set before CUDA initialises).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

N = 512
LEVELS = 6
NORMS = (1, 2)
WORKLOAD = 2  # synth recipe: ellipses + smoothed noise texture
METRIC = "W1 solves/s at 512^2 (rel 1e-4); PDHG HBM GB/s vs peak; p50/p99 latency"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def pair_ids(rank: int, step: int, batch: int):
    """Seeds of the pairs a rank solves in a step: disjoint across ranks and
    steps (replicas: each GPU works on its own pairs, nothing is exchanged)."""
    return [rank * 100000 + step * batch + k for k in range(batch)]


def reduce_max(dist, x: float, device) -> float:
    """Max of a per-rank scalar over all ranks (the job's wall time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# eps_L of eq. stop_tol at h = 1/N, scaled per ground norm, and the alpha of the
# level schedule: the library's calibrated schedule (w1_options.schedule = 1),
# copied here for the oracle arm, which runs without the library.  They are
# calibrated against the converged values of tests/golden/converged_512.json
# (bench.py --only tol-sweep): the fastest setting whose worst error over the
# calibration pairs 0-7 is at most 2.5e-5, four times below 1e-4.
TOL_SCALE = {1: 30.0, 2: 3.0}
ALPHA = {1: 0.5, 2: -1.0}  # eps_l = eps_L (h_l / h)^alpha (eq. tol_formula_propose)
THETA = {1: 1.0, 2: 1.0}   # mu tau = (theta / ||A_h||)^2 (eq. primaldual; 1/2 the paper's, 1 its footnote's)
RATIO = {1: 1.0, 2: 0.02}  # tau / mu (1: mu = tau, the paper's)
CHECK_EVERY = 64  # steps between stop tests under the calibrated schedule (the library's default there)


def stop_tol(n: int, norm: int) -> float:
    # the calibrated schedule keeps eps_L at its 512^2 value on coarser grids
    return 1e-6 / 128 * min((512.0 / n) ** 2, 1.0) * TOL_SCALE[norm]


def _oracle_solve(spec):
    """One whole Algorithm-3 solve by the FP64 oracle (a spawned worker)."""
    import oracle
    import synth
    k, norm, n, levels = spec
    r0, r1 = synth.pair(WORKLOAD, k, n=n)
    _, _, d0, d1 = synth.to_f32_pair(r0, r1)
    t0 = time.perf_counter()
    res = oracle.multilevel(d0, d1, levels=levels, norm=norm, tol=stop_tol(n, norm), alpha=ALPHA[norm],
                            theta=THETA[norm], ratio=RATIO[norm], stop=oracle.STOP_FPR, check_every=CHECK_EVERY)
    return norm, time.perf_counter() - t0, res.status


def oracle_whole_solves(seeds, n=N, levels=LEVELS, workers=None):
    """Whole Algorithm-3 solves of the given pairs, both norms, by the FP64
    oracle as it stands, at the benchmark's stop rule, one spawned process per
    host core all at once (independent pairs are the oracle's natural
    parallelism).  Returns (solves/s of the host, cores, mean seconds per solve
    for each norm, sample text)."""
    import multiprocessing as mp

    import oracle  # builds the oracle library once, before the workers load it
    oracle._load()
    workers = workers or os.cpu_count() or 1
    jobs = [(k, norm, n, levels) for norm in NORMS for k in seeds]  # p = 1 (the long solves) first
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_oracle_solve, [(seeds[0], 2, 16, 1)] * workers)  # start every worker
        t0 = time.perf_counter()
        res = pool.map(_oracle_solve, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    per = {f"L{nm}": float(np.mean([t for x, t, _ in res if x == nm])) for nm in NORMS}
    sample = (f"{len(jobs)} whole Algorithm-3 solves ({len(seeds)} pairs x {len(NORMS)} norms, {n}^2, {levels} levels, "
              f"the benchmark's stop rule) of pairs {seeds[0]}..{seeds[-1]} (the GPU arm's first timed pairs), "
              f"{workers} processes at once; value = solves / wall time")
    return len(jobs) / wall, workers, per, sample


def oracle_cost_pdhg(norm_list, budget_s=12.0):
    """Seconds per FP64 oracle solve with Algorithm 4 for each norm: whole
    solves of the bench's first pair, repeated while the budget lasts."""
    import synth
    from oracle import pdhg

    r0, r1 = synth.pair(WORKLOAD, 0)
    _, _, d0, d1 = synth.to_f32_pair(r0, r1)
    per_norm, sample = {}, []
    for norm in norm_list:
        t0, k = time.perf_counter(), 0
        while True:
            pdhg.multilevel(d0, d1, levels=LEVELS, norm=norm)
            k += 1
            if time.perf_counter() - t0 > budget_s / (2 * len(norm_list)):
                break
        per_norm[norm] = (time.perf_counter() - t0) / k
        sample.append(f"p{norm}: {k} whole solves of pair 0")
    return per_norm, "; ".join(sample)


def run_reference(args):
    """The FP64 oracle as the reference arm: whole solves of the GPU arm's
    first timed pairs at the same stop rule, on every host core.  One sample
    (one solve per pair and norm) covers the run; ms_per_step is the time of
    that sample divided by the number of steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    seeds = pair_ids(0, args.warmup, args.batch)[:max(1, min(cores, args.batch))]
    n = args.ref_n
    levels = max(1, min(LEVELS, int(np.log2(n)) - 3))
    value, cores, per, sample = oracle_whole_solves(seeds, n=n, levels=levels, workers=cores)
    wall = len(seeds) * len(NORMS) / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"ellipse_texture_{n}x{n}_pairs_{levels}_levels_both_norms", "grid": [n, n],
                   "levels": levels, "norms": ["L1", "L2"],
                   "stop": "FPR R^k < eps_l, eps_L of eq. stop_tol x " + str(TOL_SCALE) + ", alpha " + str(ALPHA)
                           + ", theta " + str(THETA) + ", tau / mu " + str(RATIO),
                   "estimate": "saddle value (Lagrangian of eq. minmax_cp)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "seconds_per_solve": per},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _gen_pair(spec):
    """One synthetic pair as float32 arrays (runs in a spawned worker process)."""
    import synth
    workload, k, n = spec
    r0, r1 = synth.pair(workload, k, n=n)
    return np.asarray(r0, dtype=np.float32), np.asarray(r1, dtype=np.float32)


def gen_pairs(specs, world=1):
    """Generate (workload, seed, side) pairs on the host cores, before CUDA starts
    (workers are spawned, never forked)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = max(1, min(32, (os.cpu_count() or 1) // max(1, world)))
    if workers == 1 or len(specs) < 8:
        return [_gen_pair(x) for x in specs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_pair, specs, chunksize=max(1, len(specs) // (4 * workers))))


# bytes a solve reads back to the host per pair: the plan's device control
# block (struct Ctl of w1_internal.h: counters and flags, masses, per-level
# steps, R^k, flags and start times, the final statistics)
CTL_BYTES = 560


def load_converged(n=N, workload=WORKLOAD):
    """The stored converged values (tests/golden/converged_512.json, or
    converged_w<workload>_<n>.json for other grids, written by
    oracle/make_converged_table.py from the FP64 oracle and the exact LP)."""
    name = "converged_512.json" if (n, workload) == (N, WORKLOAD) else f"converged_w{workload}_{n}.json"
    path = os.path.join(ROOT, "tests", "golden", name)
    try:
        with open(path) as f:
            t = json.load(f)
    except OSError:
        return None
    return {norm: {int(k): float(v["w1"]) for k, v in t.get(f"L{norm}", {}).items()} for norm in NORMS}


def run_gpu(args):
    rank, world, local = dist_env()
    B = args.batch
    DEPTH = 2 if (args.mode == "lanes" and args.pipeline) else 1
    total_steps = args.warmup + args.steps
    conv = load_converged() if (rank == 0 and args.algorithm == 3) else None
    acc_ids = sorted(set(conv[1]) | set(conv[2])) if conv else []
    # distinct pairs per step and rank (and the reference pairs), generated before CUDA starts
    specs = [(WORKLOAD, k, N) for s in range(total_steps) for k in pair_ids(rank, s, B)]
    gen = gen_pairs(specs + [(WORKLOAD, k, N) for k in acc_ids], world)
    acc_pairs = gen[len(specs):]

    import torch

    from paper_1810_00118_gb300 import w1

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    stream = torch.cuda.current_stream()
    # inputs resident in HBM before timing (and pinned host copies for the e2e run)
    host_pairs, dev_pairs = [], []
    for s in range(total_steps):
        r = gen[s * B:(s + 1) * B]
        a0 = np.ascontiguousarray(np.stack([x[0] for x in r]), dtype=np.float32)
        a1 = np.ascontiguousarray(np.stack([x[1] for x in r]), dtype=np.float32)
        host_pairs.append((torch.from_numpy(a0).pin_memory(), torch.from_numpy(a1).pin_memory()))
        dev_pairs.append((torch.from_numpy(a0).cuda(), torch.from_numpy(a1).cuda()))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    every = (w1.OK, w1.ERR_NOT_CONVERGED, w1.ERR_TIMEOUT, w1.ERR_MASS)  # read every result; only OK counts
    tol = {norm: (stop_tol(N, norm) if args.algorithm == 3 else 0.0) for norm in NORMS}

    def new_plan(norm, batch=1, tune=None):
        # Algorithm 3: the calibrated schedule (tol <= 0: its eps_L scale and alpha)
        return w1.Plan(N, N, levels=LEVELS, norm=norm, tol=0.0, batch=batch, eager=int(args.eager),
                       algorithm=args.algorithm, check_every=args.check_every, schedule=int(args.algorithm == 3),
                       tune=args.tune if tune is None else tune)

    if args.mode == "lockstep":
        # one batched plan per norm: every launch advances all B pairs together
        plans = {norm: new_plan(norm, batch=B, tune=0) for norm in NORMS}
    else:
        # lanes: one plan and one stream per pair, all enqueued asynchronously, so
        # every pair moves through its levels at its own pace and the kernels of
        # different pairs overlap on the device
        # (--lane-batch g > 1: each lane is a batched plan of g pairs)
        G = args.lane_batch
        if G < 1 or B % G:
            raise SystemExit("--lane-batch must divide --batch")
        nlane = B // G
        # pipelined steps: step s + 1 is enqueued before step s is collected, so
        # lanes that finish early start on the next step's pairs; two sets of
        # plans (and of result events) alternate between consecutive steps
        plans = {norm: [[new_plan(norm, batch=G) for _ in range(nlane)] for _ in range(DEPTH)] for norm in NORMS}
        lanes = {norm: [torch.cuda.Stream() for _ in range(nlane)] for norm in NORMS}
        done_ev = {norm: [[torch.cuda.Event(enable_timing=True) for _ in range(nlane)] for _ in range(DEPTH)]
                   for norm in NORMS}
    pair_ms = []
    ready_ev = [torch.cuda.Event(enable_timing=True) for _ in range(DEPTH)]
    pending = {}

    def submit(s, pair_set=None):
        q = s % DEPTH
        flush.fill_(float(s))
        t0, t1 = dev_pairs[s] if pair_set is None else pair_set
        if args.mode == "lockstep":
            out = []
            for norm in NORMS:
                v, st, ps, _ = plans[norm].solve_batch(t0, t1, stream=stream, allow=every)
                out.append((v, st, ps))
            pending[s] = out
            return
        ready_ev[q].record(stream)
        for norm in NORMS:
            for b in range(nlane):
                lanes[norm][b].wait_event(ready_ev[q])
                if G == 1:
                    plans[norm][q][b].solve_async(t0[b], t1[b], stream=lanes[norm][b])
                else:
                    plans[norm][q][b].solve_async(t0[b * G:(b + 1) * G], t1[b * G:(b + 1) * G],
                                                  stream=lanes[norm][b])
                done_ev[norm][q][b].record(lanes[norm][b])

    def collect(s):
        if args.mode == "lockstep":
            return pending.pop(s)
        q = s % DEPTH
        out = []
        for norm in NORMS:
            vals, sts, pss = [], [], []
            for b in range(nlane):
                done_ev[norm][q][b].synchronize()
                v, st, ps, _ = plans[norm][q][b].results(allow=every)
                vals.extend(v)
                sts.extend(st)
                pss.extend(ps)
                pair_ms.extend([ready_ev[q].elapsed_time(done_ev[norm][q][b])] * G)
            out.append((vals, sts, pss))
        return out

    def join_lanes(s):
        # the launching stream waits for every lane (their earlier work is ordered before)
        if args.mode != "lockstep":
            for norm in NORMS:
                for b in range(nlane):
                    stream.wait_event(done_ev[norm][s % DEPTH][b])

    def run_steps(first, last, out=None, step_ms=None):
        """Steps first .. last - 1, step s + 1 submitted before step s is collected."""
        t_sub = {}
        for s in range(first, last):
            t_sub[s] = time.perf_counter()
            submit(s)
            if s - first >= DEPTH - 1 and DEPTH > 1 and s > first:
                r = collect(s - 1)
                if out is not None:
                    out.append(r)
                if step_ms is not None:
                    step_ms.append((time.perf_counter() - t_sub[s - 1]) * 1e3)
            elif DEPTH == 1:
                r = collect(s)
                if out is not None:
                    out.append(r)
                if step_ms is not None:
                    step_ms.append((time.perf_counter() - t_sub[s]) * 1e3)
        if DEPTH > 1 and last > first:
            r = collect(last - 1)
            if out is not None:
                out.append(r)
            if step_ms is not None:
                step_ms.append((time.perf_counter() - t_sub[last - 1]) * 1e3)
        join_lanes(last - 1)

    def level_launches(p, k):
        # resident: one launch; streaming: one per step (path 2) or per 4 steps
        # (path 3, temporal blocking), plus one decide kernel per K steps
        if p == 1:
            return 1
        K = args.check_every or 32
        return (k if p == 2 else k // 4) + k // K

    def launches(sts):
        # prep 2, restrictions, level starts, prolongations, final 2, and the levels
        # (for a batched plan: those of the slowest pair)
        st = sts[0]
        per = 2 + (st.levels - 1) + st.levels + (st.levels - 1) + 2
        def group(g):
            return per + sum(level_launches(p, max(x.iters[lvl] for x in g)) for lvl, p in enumerate(st.path))
        if args.mode == "lockstep":
            return group(sts)
        G = args.lane_batch
        return sum(group(sts[k:k + G]) for k in range(0, len(sts), G))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(dist, x, "cuda")

    run_steps(0, args.warmup)
    barrier()
    pair_ms.clear()
    results = []
    step_ms = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        ev0.record(stream)
        run_steps(args.warmup, total_steps, out=results, step_ms=step_ms)
        ev1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    # device time on the launching stream (every lane joins it), max over ranks
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    wall = max_over_ranks(wall)
    n_ok = sum(1 for step in results for _, _, pss in step for x in pss if x == w1.OK)
    not_ok = sum(1 for step in results for _, _, pss in step for x in pss if x != w1.OK)
    solves = max_over_ranks(float(n_ok)) * world if world > 1 else n_ok
    value = solves / elapsed
    n_launch = sum(launches(sts) for step in results for _, sts, _ in step)
    pair_lat = list(pair_ms)

    # end to end through the C ABI with host buffers: w1_solve_host (host
    # densities in pinned memory, copies to the device, the solve and the W1
    # read-back inside the call), one plan and stream per pair as above, the
    # calls issued from host threads (the binding releases the GIL in the call)
    e2e = None
    if not args.no_e2e and args.mode == "lanes" and G == 1:
        import concurrent.futures as cf
        jobs = [(norm, b) for norm in NORMS for b in range(nlane)]
        nthr = min(len(jobs), args.e2e_threads)
        host_np = [(h0.numpy(), h1.numpy()) for h0, h1 in host_pairs]

        def worker(tid, steps, out):
            # a thread's pairs of every step back to back: no barrier between
            # steps (each step's inputs, 2 B MiB per norm, exceed L2 already)
            for s in steps:
                for norm, b in jobs[tid::nthr]:
                    v, st, status = plans[norm][0][b].solve_host(host_np[s][0][b], host_np[s][1][b],
                                                                 stream=lanes[norm][b], allow=every)
                    out.append(status)

        def e2e_run(steps, ex):
            outs = [[] for _ in range(nthr)]
            list(ex.map(lambda t: worker(t, steps, outs[t]), range(nthr)))
            return [x for o in outs for x in o]

        with cf.ThreadPoolExecutor(max_workers=nthr) as ex:
            e2e_run([0], ex)  # warm-up: the plans' input buffers
            flush.fill_(0.0)
            torch.cuda.synchronize()
            barrier()
            t0e = time.perf_counter()
            sts_e2e = [e2e_run(range(args.warmup, total_steps), ex)]
            barrier()
            e2e_wall = max_over_ranks(time.perf_counter() - t0e)
        ok_e2e = sum(1 for st_ in sts_e2e for x in st_ if x == w1.OK)
        e2e = {"value": (ok_e2e * world) / e2e_wall, "unit": "solves/s",
               "h2d_bytes_per_step": 2 * N * N * 4 * B * len(NORMS),
               "d2h_bytes_per_step": CTL_BYTES * B * len(NORMS),
               "path": f"w1_solve_host (C ABI, host densities in pinned memory) from {nthr} host threads, one plan "
                       "and stream per pair; each thread runs its pairs of every timed step back to back (no "
                       "barrier between steps; a step's inputs exceed L2); wall clock around all of them",
               "not_ok": sum(1 for st_ in sts_e2e for x in st_ if x != w1.OK)}

    # accuracy: the reference pairs solved by the same plans (lanes) and compared
    # with their stored converged values (FP64 oracle / exact LP)
    accuracy = None
    if conv and acc_ids and args.mode == "lanes" and G == 1 and not args.no_accuracy:
        a0 = torch.from_numpy(np.stack([x[0] for x in acc_pairs])).cuda()
        a1 = torch.from_numpy(np.stack([x[1] for x in acc_pairs])).cuda()
        errs, prim, sts_acc = {}, {}, {}
        for norm in NORMS:
            e, pe, ss = [], [], []
            for i, k in enumerate(acc_ids):
                if k not in conv[norm]:
                    continue
                p = plans[norm][0][i % nlane]
                p.solve_async(a0[i], a1[i], stream=lanes[norm][i % nlane])
                lanes[norm][i % nlane].synchronize()
                v, st, ps, _ = p.results(allow=every)
                ref = conv[norm][k]
                e.append(abs(v[0] - ref) / ref)
                pe.append(abs(st[0].primal - ref) / ref)
                ss.append(ps[0])
            errs[f"L{norm}"], prim[f"L{norm}"], sts_acc[f"L{norm}"] = e, pe, ss
        accuracy = {"max_rel_err_vs_converged": {k: (float(max(v)) if v else None) for k, v in errs.items()},
                    "rel_err_vs_converged": errs,
                    "primal_max_rel_err_vs_converged": {k: (float(max(v)) if v else None) for k, v in prim.items()},
                    "pairs": {f"L{n}": sorted(conv[n]) for n in NORMS}, "statuses": sts_acc,
                    "reference": "tests/golden/converged_512.json (p = 1: exact LP; p = 2: FP64 oracle at "
                                 "eps_L / 1e4), written by oracle/make_converged_table.py",
                    "what": "reported W1 (saddle value) of each reference pair against its converged value; "
                            "primal: f(m) of the same solves"}

    # secondary: the paper's own schedule (eq. stop_tol, alpha = -1, theta = 1/2)
    # for the same pairs and lanes: throughput and the reference pairs' errors
    paper = None
    if args.paper_steps > 0 and args.mode == "lanes" and G == 1 and args.algorithm == 3:
        pp = {norm: [w1.Plan(N, N, levels=LEVELS, norm=norm, batch=1) for _ in range(nlane)] for norm in NORMS}

        def paper_step(s):
            flush.fill_(float(s))
            t0_, t1_ = dev_pairs[s]
            ready_ev[0].record(stream)
            for norm in NORMS:
                for b in range(nlane):
                    lanes[norm][b].wait_event(ready_ev[0])
                    pp[norm][b].solve_async(t0_[b], t1_[b], stream=lanes[norm][b])
                    done_ev[norm][0][b].record(lanes[norm][b])
            sts_ = []
            for norm in NORMS:
                for b in range(nlane):
                    done_ev[norm][0][b].synchronize()
                    sts_.extend(pp[norm][b].results(allow=every)[2])
                    stream.wait_event(done_ev[norm][0][b])
            return sts_

        paper_step(0)
        barrier()
        e0p, e1p = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0p.record(stream)
        sts_p = [paper_step(args.warmup + s) for s in range(min(args.paper_steps, args.steps))]
        e1p.record(stream)
        barrier()
        n_ok_p = sum(1 for x in sts_p for y in x if y == w1.OK)
        paper = {"solves_per_s": n_ok_p / (e0p.elapsed_time(e1p) / 1e3), "steps": len(sts_p),
                 "schedule": "eq. stop_tol eps_L, alpha -1, theta 1/2 (the paper's; w1_options.schedule = 0)"}
        if conv and acc_ids:
            a0p = torch.from_numpy(np.stack([x[0] for x in acc_pairs])).cuda()
            a1p = torch.from_numpy(np.stack([x[1] for x in acc_pairs])).cuda()
            errs_p = {}
            for norm in NORMS:
                e = []
                for i, k in enumerate(acc_ids):
                    if k not in conv[norm]:
                        continue
                    p = pp[norm][i % nlane]
                    p.solve_async(a0p[i], a1p[i], stream=lanes[norm][i % nlane])
                    lanes[norm][i % nlane].synchronize()
                    e.append(abs(p.results(allow=every)[0][0] - conv[norm][k]) / conv[norm][k])
                errs_p[f"L{norm}"] = float(max(e)) if e else None
            paper["max_rel_err_vs_converged"] = errs_p
        for norm in NORMS:
            for p in pp[norm]:
                p.close()

    # latency of one solve with the GPU otherwise idle: one pair at a time through
    # the blocking entry point, CUDA events around each solve
    solo = {}
    tuned = args.algorithm == 3  # the latency-tuned plan (tune = 1) beside the default one
    for norm in (NORMS if args.solo > 0 else ()):
        for tune in ((0, 1) if tuned else (0,)):
            with new_plan(norm, tune=tune) as p1:
                ts = []
                for k in range(args.solo):
                    t0s, t1s = dev_pairs[k % total_steps][0][k % B], dev_pairs[k % total_steps][1][k % B]
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    p1.solve(t0s, t1s, stream=stream, allow=every)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
            solo[f"L{norm}" + ("_latency_tuned" if tune else "")] = {
                "p50": float(np.percentile(ts, 50)), "p99": float(np.percentile(ts, 99)), "pairs": len(ts)}
    solo["what"] = ("one solve with the GPU otherwise idle (w1_solve, CUDA events); _latency_tuned: the plan's "
                    "kernels picked by the autotuner for one solve alone (tune = 1)")

    for p in plans.values():
        for q in (p if isinstance(p, list) else [p]):
            for r in (q if isinstance(q, list) else [q]):
                r.close()
    torch.cuda.synchronize()

    # rooflines (the dominant on-chip kernel; the streaming kernels at 8192^2)
    roof = None
    if not args.no_roofline:
        roof = roofline(w1, torch, stream, args)

    # serving (Poisson arrivals of mixed sizes) and the mixed-size batch, short
    serving = mixed = None
    if rank == 0 and not args.no_extras and args.algorithm == 3:
        serving = serve_summary(w1, torch, args)
        mixed = mixed_summary(w1, torch, args)

    line = None
    if rank == 0:
        lat = np.array(step_ms) / len(NORMS)
        iters = {f"L{n}": results[-1][i][1][0].iters for i, n in enumerate(NORMS)}
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 iterates, compensated f64 reductions",
            "data": "synthetic",
            "config": {"workload": "ellipse_texture_512x512_pairs_6_levels_both_norms", "grid": [N, N],
                       "levels": LEVELS, "norms": ["L1", "L2"],
                       "algorithm": {3: "Algorithm 3 (multilevel Chambolle-Pock)",
                                     4: "Algorithm 4 (multilevel prox-PDHG)"}[args.algorithm],
                       "stop": ("FPR R^k < eps_l (eq. pd_stop), eps_l = eps_L (h_l/h)^alpha, eps_L of eq. stop_tol x "
                                "scale; the calibrated schedule (w1_options.schedule = 1): scale "
                                + json.dumps({f"L{k}": v for k, v in TOL_SCALE.items()}) + ", alpha "
                                + json.dumps({f"L{k}": v for k, v in ALPHA.items()}) + ", theta "
                                + json.dumps({f"L{k}": v for k, v in THETA.items()}) + ", tau / mu "
                                + json.dumps({f"L{k}": v for k, v in RATIO.items()})
                                + f", tested every {args.check_every or CHECK_EVERY} steps")
                       if args.algorithm == 3 else "eq. stop_tol for Algorithm 4",
                       "tol": {f"L{k}": v for k, v in tol.items()},
                       "estimate": "saddle value: Lagrangian of eq. minmax_cp at the returned pair",
                       "batch_per_norm": B, "mode": args.mode,
                       "pairs_per_lane": args.lane_batch if args.mode == "lanes" else B,
                       "l2": "flushed before every step (256 MiB write, inside the timed region); each step's "
                             "inputs (2 x B x 1 MiB) are larger than L2 as well",
                       "pipelined_steps": DEPTH if args.mode == "lanes" else 1,
                       "parallelism": f"replicas x{world}"},
            "timer": {"kind": "CUDA events on the launching stream, every lane joined to it", "wall_s": wall},
            "solves_counted": "status W1_OK only", "not_ok": not_ok,
            "max_rel_err_vs_converged": accuracy["max_rel_err_vs_converged"] if accuracy else None,
            "accuracy": accuracy,
            "paper_schedule": paper,
            "batch_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                 "what": "one step (B pairs, both norms) / 2, submit to W1 values on the host "
                                         "(with pipelined steps the next step is already running meanwhile)"},
            "solo_latency_ms": solo,
            "pair_latency_ms": ({"p50": float(np.percentile(pair_lat, 50)), "p99": float(np.percentile(pair_lat, 99)),
                                 "what": "per pair: its step's submission to the end of its solve on its "
                                         "stream (CUDA events)"}
                                if pair_lat else None),
            "serving": serving,
            "mixed": mixed,
            "iters_first_pair": iters,
            "gpu_launches": n_launch,
            "e2e": e2e,
            "roofline": roof,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline and args.algorithm == 4:
            per_norm, sample = oracle_cost_pdhg(NORMS, budget_s=args.ref_budget)
            line["cpu_baseline"] = {"value": len(NORMS) / sum(per_norm.values()), "unit": "solves/s", "cores": 1,
                                    "kind": "oracle", "sample": "FP64 prox-PDHG oracle (numpy, one thread): " + sample}
        elif not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            seeds = pair_ids(0, args.warmup, B)[:min(cores, B)]
            cpu_v, cores, per, sample = oracle_whole_solves(seeds, workers=cores)
            line["cpu_baseline"] = {"value": cpu_v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                    "sample": sample, "seconds_per_solve": per}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ncu DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum), from
# the captures summarised under profiles/ (taken with the current kernels); None
# where no capture of the current kernel exists.  Streaming kernels: captured at
# 4096^2 and scaled by 4 to 8192^2 (their traffic grows with the number of nodes);
# k_resident4: the 256^2 level on 16 CTAs, p = 2, 2000 steps per launch.
TRAFFIC = {"k_step": 4 * 441.28e6, "k_tblock": 4 * 431.0e6, "k_resident4": 1102592.0}

FP32_LANES_PER_SM = 128  # FP32 units per SM; two flops per FMA
SM_MAX_MHZ = 2070.0
FLOPS_PER_NODE_STEP = {1: 25, 2: 30, 3: 30}  # eq. primaldual: gradient, shrink, extrapolation, divergence, dual step


def _time_steps(w1, torch, stream, rho, h, norm, mu, path, a, b, cluster=0):
    """Time per step from two runs of a and b steps (the difference removes the
    fixed cost of a call: allocation and the load and store of the level)."""
    n = rho.shape[0]
    kw = {"cluster": cluster} if path == 1 else {}
    ms = []
    for k in (a, b):
        m1, m2, phi = (torch.zeros((n, n), device="cuda") for _ in range(3))
        w1.cp_steps(rho, m1, m2, phi, h, norm, mu, mu, 8 if path != 1 else 32, path=path, stream=stream, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        w1.cp_steps(rho, m1, m2, phi, h, norm, mu, mu, k, path=path, stream=stream, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        del m1, m2, phi
    return (ms[1] - ms[0]) / (b - a)


def roofline(w1, torch, stream, args):
    """Rooflines, timed with CUDA events on the launching stream.

    resident (the dominant kernel of a solve: the on-chip level solve, here a
    256^2 level in a 16-CTA cluster, p = 2): arithmetic of eq. primaldual per
    node and step against the FP32 rate of the SMs the launch occupies (its
    limit in practice is instruction issue and the two cluster barriers per step).
    streaming: one step per launch on an 8192^2 grid (1.9 GB, far above L2),
    28 algorithmic bytes per node and step against the measured HBM copy rate.
    temporal_blocking: 4 steps per launch on chip; its figure is effective
    bandwidth (28 B per node-step), not DRAM traffic."""
    peak, kind = peaks()
    out = {}
    n = args.roof_n
    h = 1.0 / n
    rho = torch.randn((n, n), device="cuda") * 0.1
    rho -= rho.mean()
    mu = float(np.float32(0.5 * h / (2 * np.sqrt(2.0))))
    for path, key, name in ((2, "k_step", "k_step (one step per launch)"),
                            (3, "k_tblock", "k_tblock (temporal blocking, 4 steps per launch)")):
        ms_step = _time_steps(w1, torch, stream, rho, h, 1, mu, path, 16, 16 + args.roof_iters)
        per_launch = 4 if path == 3 else 1
        achieved = 28.0 * n * n / (ms_step * 1e-3) / 1e9
        out[key] = {"kernel": name, "grid": [n, n], "bound": "hbm", "achieved": achieved, "peak": peak,
                    "peak_kind": kind, "unit": "GB/s", "frac": achieved / peak, "traffic": TRAFFIC[key],
                    "ms_per_launch": ms_step * per_launch, "steps_per_launch": per_launch,
                    "algorithmic_bytes_per_launch": 28 * n * n * per_launch}
    out["k_tblock"]["note"] = ("effective bandwidth, not DRAM traffic: 28 B per node-step; the tile and its "
                               "halo are read once per 4 steps")
    del rho
    # the dominant kernel of the benchmark's solves (launch list: the p = 2 cluster
    # levels, 128^2 and 256^2, 35 % of the device time): the 256^2 level on 16 CTAs
    nr, kr, nm = 256, 2000, 2
    hr = 1.0 / nr
    rr = torch.randn((nr, nr), device="cuda") * 0.1
    rr -= rr.mean()
    mur = float(np.float32(0.5 * hr / (2 * np.sqrt(2.0))))
    ms_step = _time_steps(w1, torch, stream, rr, hr, nm, mur, 1, 256, 256 + kr, cluster=16)
    flops_step = FLOPS_PER_NODE_STEP[nm] * nr * nr
    fpeak = 16 * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops_step / (ms_step * 1e-3) / 1e12
    res = {"kernel": "k_resident4 (on-chip level solve, 256^2 level, cluster of 16 CTAs, p = 2)", "grid": [nr, nr],
           "bound": "alu", "achieved": achieved, "peak": fpeak,
           "peak_kind": "derived: 16 SMs x 128 FP32 lanes x 2 flops x 2070 MHz", "unit": "TFLOP/s",
           "frac": achieved / fpeak, "traffic": TRAFFIC["k_resident4"], "us_per_step": ms_step * 1e3,
           "steps_per_launch": kr, "flops_per_node_step": FLOPS_PER_NODE_STEP[nm],
           "note": "issue and barrier-latency bound: no HBM traffic per step; traffic is per launch of "
                   f"{kr} steps (the level is loaded once)"}
    # the same per-step time against 28 algorithmic bytes per node and step (the
    # measure of the streaming kernels; this level is on chip, so it is not DRAM traffic)
    res["bytes_per_node_step"] = 28
    res["achieved_alg_GBps"] = 28.0 * nr * nr / (ms_step * 1e-3) / 1e9
    res["frac_alg_bytes_vs_hbm"] = res["achieved_alg_GBps"] / peak
    del rr
    # the wide on-chip kernel: the 512^2 level on a 16-CTA cluster
    nw = 512
    hw = 1.0 / nw
    rw = torch.randn((nw, nw), device="cuda") * 0.1
    rw -= rw.mean()
    muw = float(np.float32(0.5 * hw / (2 * np.sqrt(2.0))))
    msw = _time_steps(w1, torch, stream, rw, hw, nm, muw, 1, 64, 64 + 500, cluster=16)
    res["wide"] = {"kernel": "k_resident_wide (512^2 level, cluster of 16 CTAs, p = 2)", "us_per_step": msw * 1e3,
                   "achieved_alg_GBps": 28.0 * nw * nw / (msw * 1e-3) / 1e9,
                   "frac_alg_bytes_vs_hbm": 28.0 * nw * nw / (msw * 1e-3) / 1e9 / peak,
                   "achieved_TFLOPs": FLOPS_PER_NODE_STEP[nm] * nw * nw / (msw * 1e-3) / 1e12,
                   "frac_alu": FLOPS_PER_NODE_STEP[nm] * nw * nw / (msw * 1e-3) / 1e12 / fpeak}
    res["streaming"] = out["k_step"]
    res["temporal_blocking"] = out["k_tblock"]
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--batch", type=int, default=128, help="pairs per norm per step")
    ap.add_argument("--lane-batch", type=int, default=1, help="lanes: pairs per lane (a batched plan per lane)")
    ap.add_argument("--pipeline", type=int, default=1, choices=[0, 1],
                    help="lanes: submit step s + 1 before collecting step s (1) or drain every step (0)")
    ap.add_argument("--mode", default="lanes", choices=["lanes", "lockstep"],
                    help="lanes: one async plan+stream per pair; lockstep: one batched plan per norm")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--roof-n", type=int, default=8192)
    ap.add_argument("--roof-iters", type=int, default=96)
    ap.add_argument("--ref-budget", type=float, default=12.0, help="Algorithm 4 CPU baseline: seconds")
    ap.add_argument("--ref-n", type=int, default=N, help="oracle arm: grid side of the whole solves")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-threads", type=int, default=128, help="e2e: host threads calling w1_solve_host")
    ap.add_argument("--no-extras", action="store_true", help="skip the short serving and mixed-batch legs")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the solves of the reference pairs")
    ap.add_argument("--paper-steps", type=int, default=2,
                    help="steps timed with the paper's own schedule beside the headline (0: skip)")
    ap.add_argument("--solo", type=int, default=8, help="pairs solved one at a time for the latency figure")
    ap.add_argument("--tune", type=int, default=0, choices=[0, 1, 2, 3],
                    help="lanes: per-level kernel choice (0 fixed rules, 1 latency, 3 SM-time; see w1_options.tune)")
    ap.add_argument("--check-every", type=int, default=0,
                    help="steps between stop tests (multiple of 8; 0: the library's default, 64 for Algorithm 3 "
                         "under the calibrated schedule, 8 for Algorithm 4)")
    ap.add_argument("--algorithm", type=int, default=3, choices=[3, 4],
                    help="3: multilevel Chambolle-Pock (the headline); 4: multilevel prox-PDHG")
    ap.add_argument("--eager", action="store_true",
                    help="launch level kernels directly (no CUDA graph) so profilers see every kernel")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000", help="serving: arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=400, help="serving: requests per rate (at least)")
    ap.add_argument("--min-seconds", type=float, default=0.0, help="serving: at least rate*this requests")
    ap.add_argument("--slots", type=int, default=48, help="serving: solves in flight")
    ap.add_argument("--serve-batch", type=int, default=1, help="serving: pairs a slot solves together")
    ap.add_argument("--latency-below", type=int, default=4,
                    help="serving: in-flight count below which requests get latency-tuned slots (0: off)")
    ap.add_argument("--only", default="solve",
                    choices=["solve", "stream-kernel", "tblock-kernel", "resident-kernel", "pdhg-kernel", "serve",
                             "mixed", "tol-sweep", "solve3d", "3d-kernel", "cascade-vs-single"],
                    help="kernel-only runs for profiling: one level's steps through w1_cp_steps")
    ap.add_argument("--kn", type=int, default=256, help="grid side for --only *-kernel")
    ap.add_argument("--sweep-size", type=int, default=0, help="--only tol-sweep: grid side (0: 512)")
    ap.add_argument("--kiters", type=int, default=1000, help="steps for --only *-kernel")
    ap.add_argument("--knorm", type=int, default=1)
    ap.add_argument("--kcluster", type=int, default=0, help="--only resident-kernel: CTAs per level (0: auto)")
    ap.add_argument("--kpath3", type=int, default=2, choices=[2, 3],
                    help="--only 3d-kernel: 2 two launches per step, 3 one launch per step")
    ap.add_argument("--n3", type=int, default=64, help="--only solve3d: grid side of the 3-D solves")
    ap.add_argument("--pairs3", type=int, default=8, help="--only solve3d: pairs per norm")
    ap.add_argument("--roof-n3", type=int, default=256, help="--only solve3d: grid side of the step-kernel timing")
    ap.add_argument("--mixed-norm", type=int, default=2, help="mixed-size batch: ground norm")
    ap.add_argument("--mixed-schedule", type=int, default=1, choices=[0, 1],
                    help="mixed-size batch: level tolerances (1 the calibrated schedule, 0 the paper's)")
    ap.add_argument("--mixed-modes", default="loop,lanes,lockstep,lockstep-tuned,persistent")
    ap.add_argument("--mixed-spec", default="", help="mixed-size batch override, e.g. 64:128,128:96")
    ap.add_argument("--mixed-passes", type=int, default=2, help="default line: timed passes of the mixed batch")
    ap.add_argument("--serve-summary", default="30:300,300:2000",
                    help="default line: serving rates and request counts, rate:requests,...")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only == "serve":
        return run_serve(args)
    if args.only == "mixed":
        return run_mixed(args)
    if args.only == "tol-sweep":
        return run_tol_sweep(args)
    if args.only == "solve3d":
        return run_solve3d(args)
    if args.only == "cascade-vs-single":
        return run_cascade_vs_single(args)
    if args.only != "solve":
        return run_kernel_only(args)
    return run_gpu(args)


# Mixed-size batch: (grid side, pairs, levels 16 -> side), Gaussian-mixture densities
MIXED = ((64, 128, 3), (128, 96, 4), (256, 32, 5))


def run_mixed(args):
    """256 pairs of three grid sizes solved per step, in several ways: a loop of
    single solves (one at a time), lanes (one async single-pair plan and stream
    per pair), lockstep (one batched plan per size, the three on their own
    streams), and lockstep with per-level kernels chosen by the autotuner
    (throughput objective).  Times with CUDA events on the launching stream."""
    import torch

    import synth
    from paper_1810_00118_gb300 import w1

    torch.cuda.set_device(0)
    norm = args.mixed_norm
    stream = torch.cuda.current_stream()
    passes = args.warmup + args.steps
    global MIXED
    if args.mixed_spec:
        # side:pairs,side:pairs,... (levels down to 16^2)
        MIXED = tuple((int(a), int(b), int(np.log2(int(a) // 16)) + 1)
                      for a, b in (x.split(":") for x in args.mixed_spec.split(",")))
    data = []  # per pass: per class (t0, t1) [B, n, n]
    for s in range(passes):
        per = []
        for ci, (n, B, _) in enumerate(MIXED):
            r = [synth.pair(3, 100000 * s + 1000 * ci + k, n=n) for k in range(B)]
            a0 = np.ascontiguousarray(np.stack([x[0] for x in r]), dtype=np.float32)
            a1 = np.ascontiguousarray(np.stack([x[1] for x in r]), dtype=np.float32)
            per.append((torch.from_numpy(a0).cuda(), torch.from_numpy(a1).cuda()))
        data.append(per)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ok = (w1.OK, w1.ERR_NOT_CONVERGED)
    total = sum(B for _, B, _ in MIXED)
    modes = [m for m in args.mixed_modes.split(",") if m]
    out = {}
    w1_ref = None
    sch = args.mixed_schedule
    for mode in modes:
        if mode == "loop":
            plans = [w1.Plan(n, n, levels=L, norm=norm, schedule=sch) for n, _, L in MIXED]
        elif mode == "lanes":
            plans = [[w1.Plan(n, n, levels=L, norm=norm, schedule=sch) for _ in range(B)] for n, B, L in MIXED]
            lanes = [[torch.cuda.Stream() for _ in range(B)] for _, B, _ in MIXED]
        elif mode == "persistent":
            plans = w1.Mixed([(n, n, B) for n, B, _ in MIXED], norm=norm, schedule=sch)
        else:
            tune = 2 if mode == "lockstep-tuned" else 0
            plans = [w1.Plan(n, n, levels=L, norm=norm, batch=B, tune=tune, schedule=sch) for n, B, L in MIXED]
            lanes = [torch.cuda.Stream() for _ in MIXED]

        def one_pass(s):
            flush.fill_(float(s))
            vals = []
            if mode == "loop":
                for ci, (n, B, _) in enumerate(MIXED):
                    t0, t1 = data[s][ci]
                    for b in range(B):
                        v, _, _ = plans[ci].solve(t0[b], t1[b], stream=stream, allow=ok)
                        vals.append(v)
                return vals
            if mode == "persistent":
                plans.solve_async([d[0] for d in data[s]], [d[1] for d in data[s]], stream=stream)
                stream.synchronize()
                for ci in range(len(MIXED)):
                    vals.extend(plans.results(ci, allow=ok)[0])
                return vals
            ready = torch.cuda.Event()
            ready.record(stream)
            for ci, (n, B, _) in enumerate(MIXED):
                t0, t1 = data[s][ci]
                if mode == "lanes":
                    for b in range(B):
                        lanes[ci][b].wait_event(ready)
                        plans[ci][b].solve_async(t0[b], t1[b], stream=lanes[ci][b])
                else:
                    lanes[ci].wait_event(ready)
                    plans[ci].solve_async(t0, t1, stream=lanes[ci])
            for ci, (n, B, _) in enumerate(MIXED):
                if mode == "lanes":
                    for b in range(B):
                        stream.wait_stream(lanes[ci][b])
                        lanes[ci][b].synchronize()
                        vals.append(plans[ci][b].results(allow=ok)[0][0])
                else:
                    stream.wait_stream(lanes[ci])
                    lanes[ci].synchronize()
                    vals.extend(plans[ci].results(allow=ok)[0])
            return vals

        for s in range(args.warmup):
            one_pass(s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vals = [one_pass(s) for s in range(args.warmup, passes)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        flat = np.array([v for p in vals for v in p])
        if w1_ref is None:
            w1_ref = flat
        out[mode] = {"solves_per_s": args.steps * total / (ms / 1e3), "ms_per_pass": ms / args.steps,
                     "max_rel_diff_vs_first_mode": float(np.max(np.abs(flat - w1_ref) / np.abs(w1_ref)))}
        if mode == "persistent":
            out[mode]["persistent_classes"] = [plans.persistent(c) for c in range(len(MIXED))]
            out[mode]["launch"] = plans.launch_info()
            plans.close()
        del plans
        torch.cuda.synchronize()
    print(json.dumps({"only": "mixed",
                      "workload": "gauss8 mixed: " + ", ".join(f"{B} x {n}^2 ({L} levels)" for n, B, L in MIXED), "norm": norm, "pairs_per_pass": total, "passes": args.steps,
                      "l2": "flushed before every pass", "modes": out}), flush=True)
    return 0


def run_tol_sweep(args):
    """Tolerance schedule study (eq. tol_formula_propose, the alpha study of
    Sec. 6.2, the level count of Sec. 6.3) on grids with stored converged values
    (--kn: 512 for the benchmark's pairs, 128 or 256 for the serving mix's): for
    each norm, eps_l = s * eps_L (h_l / h)^alpha with eps_L of eq. stop_tol, for
    several scales s, alphas, step sizes theta (mu tau = (theta / ||A_h||)^2)
    and step ratios tau / mu; the reported W1 (saddle value) of the reference
    pairs against their converged values and the throughput of a batch of lanes
    (one plan and stream per pair, CUDA events)."""
    import torch

    import synth
    from paper_1810_00118_gb300 import w1

    n = args.sweep_size or N
    workload = WORKLOAD if n == N else 4
    conv = load_converged(n, workload)
    if not conv:
        raise SystemExit("no stored converged values for this grid")
    levels = max(1, int(np.log2(n)) - 3)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    every = (w1.OK, w1.ERR_NOT_CONVERGED, w1.ERR_TIMEOUT, w1.ERR_MASS)
    out = []
    for norm in NORMS:
        ids = sorted(conv[norm])
        if not ids:
            continue
        pairs = [synth.pair(workload, k, n=n) for k in ids]
        t0 = torch.from_numpy(np.ascontiguousarray(np.stack([p[0] for p in pairs]), dtype=np.float32)).cuda()
        t1 = torch.from_numpy(np.ascontiguousarray(np.stack([p[1] for p in pairs]), dtype=np.float32)).cuda()
        # the throughput batch: the reference pairs repeated to args.batch lanes
        B = max(args.batch, len(ids))
        lanes = [torch.cuda.Stream() for _ in range(B)]
        grid = SWEEP_GRID[norm]
        n_cal = max(1, len(ids) // 2)  # the first half calibrates, the second half is held out
        for theta, alpha, ratio, scales in grid:
            for scale in scales:
                tol = 1e-6 / 128 * (512.0 / n) ** 2 * scale
                plans = [w1.Plan(n, n, levels=levels, norm=norm, tol=tol, alpha=alpha, theta=theta,
                                 step_ratio=ratio) for _ in range(B)]
                for rep in range(2):  # first pass: graph builds; second: timed
                    ready = torch.cuda.Event()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    ready.record(stream)
                    for b in range(B):
                        lanes[b].wait_event(ready)
                        plans[b].solve_async(t0[b % len(ids)], t1[b % len(ids)], stream=lanes[b])
                        stream.wait_stream(lanes[b])
                    e1.record(stream)
                    torch.cuda.synchronize()
                errs, ok = {}, 0
                for b, p in enumerate(plans):
                    v, st, ps, _ = p.results(allow=every)
                    ok += ps[0] == w1.OK
                    if b < len(ids):
                        errs[ids[b]] = (v[0] - conv[norm][ids[b]]) / conv[norm][ids[b]]
                    p.close()
                ms = e0.elapsed_time(e1)
                cal = [abs(errs[k]) for k in ids[:n_cal]]
                held = [abs(errs[k]) for k in ids[n_cal:]]
                out.append({"n": n, "norm": norm, "levels": levels, "theta": theta, "alpha": alpha, "ratio": ratio,
                            "scale": scale, "solves_per_s": ok / (ms / 1e3), "not_ok": B - ok,
                            "max_abs_rel_err_calibration": float(max(cal)) if cal else None,
                            "max_abs_rel_err_held_out": float(max(held)) if held else None,
                            "rel_errs": {str(k): float(e) for k, e in errs.items()}})
                print(json.dumps(out[-1]), flush=True)
    print(json.dumps({"only": "tol-sweep", "grid": n, "batch": args.batch, "reference_pairs": {
        f"L{m}": sorted(conv[m]) for m in NORMS}, "rows": out}))
    return 0


# (theta, alpha, tau / mu, eps_L scales) per norm for --only tol-sweep
SWEEP_GRID = {1: [(1.0, 0.5, 1.0, (30.0, 10.0, 5.0, 3.0, 1.0))],
              2: [(1.0, -1.0, 0.02, (2.0, 1.0, 0.5, 0.25))]}


def run_cascade_vs_single(args):
    """256^2 Gaussian-mixture pairs (8 components, 1e-4 floor), p = 2: the 5-level
    cascade 16 -> 256 (Algorithm 3) against a single level started from zero
    (Algorithm 1) with the same finest-level tolerance, same GPU, one solve at a
    time (CUDA events): time per solve, finest-level steps, W1 agreement."""
    import torch

    import synth
    from paper_1810_00118_gb300 import w1

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n, norm, npairs = 256, 2, 4
    pairs = []
    for k in range(npairs):
        r0, r1 = synth.pair(1, k)
        pairs.append(tuple(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in (r0, r1)))
    out = {}
    for levels in (5, 1):
        with w1.Plan(n, n, levels=levels, norm=norm, max_iters=4_000_000) as plan:
            plan.solve(*pairs[0], stream=stream, allow=(w1.OK, w1.ERR_NOT_CONVERGED))  # warm-up (graph build)
            ms, vals, fin = [], [], []
            for a, b in pairs:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                v, st, status = plan.solve(a, b, stream=stream, allow=(w1.OK, w1.ERR_NOT_CONVERGED))
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
                vals.append(v)
                fin.append(st.iters[-1])
            out[levels] = {"levels": levels, "ms_per_solve": float(np.mean(ms)), "finest_steps": fin, "w1": vals,
                           "converged": bool(st.converged)}
        print(json.dumps(out[levels]), flush=True)
    rel = [abs(a - b) / abs(b) for a, b in zip(out[5]["w1"], out[1]["w1"])]
    print(json.dumps({"only": "cascade-vs-single", "grid": [n, n], "norm": "L2", "pairs": npairs,
                      "speedup": out[1]["ms_per_solve"] / out[5]["ms_per_solve"],
                      "finest_step_ratio": float(np.mean(out[1]["finest_steps"]) / np.mean(out[5]["finest_steps"])),
                      "max_rel_w1_diff": float(max(rel)), "cascade": out[5], "single": out[1]}))
    return 0


# Algorithmic bytes per node and step of the streamed 3-D step.  Two launches:
# m' reads m1..m3 and phi, writes m1..m3 and mbar (40 B); phi' reads mbar, rho
# and phi and writes phi (24 B).  One launch: reads m1..m3, phi and rho, writes
# m1..m3 and phi (36 B).  Neighbour reads hit cache lines already read.
BYTES3_PER_NODE_STEP = 64.0
BYTES3_ONE_LAUNCH = 36.0


def run_solve3d(args):
    """3-D workload: full Algorithm-3 solves (w1_solve3d, h^3 weights, default
    levels and tolerance) of Gaussian-mixture voxel pairs, each norm; the step
    kernels on a grid above L2 against the HBM roofline; the FP64 3-D oracle on
    the host for one pair at the same size (bounded by a step count)."""
    import torch

    import synth
    from paper_1810_00118_gb300 import w1

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n = args.n3
    pairs = [synth.pair3(n, k) for k in range(args.pairs3)]
    dev = [(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).cuda()) for a, b in pairs]
    for norm in (1, 2, 3):
        w1.solve3d(*dev[0], norm=norm, stream=stream)  # warm-up
    rows = []
    with ClockSampler(0) as clk:
        for norm in (1, 2, 3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            vals, iters, brackets = [], [], []
            torch.cuda.synchronize()
            e0.record(stream)
            for a, b in dev:
                v, st, status = w1.solve3d(a, b, norm=norm, stream=stream)
                vals.append(v)
                iters.append(st.iters)
                brackets.append((st.ub - st.lb) / max(abs(v), 1e-300))
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rows.append({"norm": norm, "solves_per_s": len(dev) / (ms / 1e3), "ms_per_solve": ms / len(dev),
                         "levels": st.levels, "iters_pair0": iters[0], "w1_pair0": vals[0],
                         "max_rel_bracket": float(max(brackets))})
            print(json.dumps(rows[-1]), flush=True)
    # step kernels above L2: 256^3 = 16.8M voxels, 1.07 GB per step
    rn = args.roof_n3
    rng = np.random.default_rng(3)
    rho = torch.from_numpy(rng.normal(size=(rn, rn, rn)).astype(np.float32)).cuda()
    rho -= rho.mean()
    st4 = [torch.zeros((rn, rn, rn), device="cuda") for _ in range(4)]
    h = 1.0 / rn
    mu = float(np.float32(0.5 * h / (2 * np.sqrt(3.0))))
    steps = 64
    peak, src = peaks()
    kern = {}
    for path, nbytes in ((2, BYTES3_PER_NODE_STEP), (3, BYTES3_ONE_LAUNCH)):
        w1.cp_steps3d(rho, *st4, h, 1, mu, mu, 4, path=path, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        w1.cp_steps3d(rho, *st4, h, 1, mu, mu, steps, path=path, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us_p = e0.elapsed_time(e1) * 1e3 / steps
        gbs_p = nbytes * rn ** 3 / (us_p * 1e-6) / 1e9
        kern[path] = {"us_per_step": us_p, "alg_bytes_per_step": nbytes * rn ** 3, "achieved_GBps": gbs_p,
                      "peak_GBps": peak, "frac": gbs_p / peak, "peak_source": src}
    us, gbs = kern[2]["us_per_step"], kern[2]["achieved_GBps"]
    # oracle on the host: one pair at the solve size, steps timed on a bounded run
    from oracle import d3
    r0, r1 = pairs[0]
    t0 = time.perf_counter()
    ref = d3.multilevel(r0.astype(np.float32).astype(np.float64), r1.astype(np.float32).astype(np.float64),
                        levels=rows[0]["levels"], norm=1, replay=rows[0]["iters_pair0"])
    cpu_s = time.perf_counter() - t0
    out = {"only": "solve3d", "grid": [n, n, n], "pairs_per_norm": len(dev), "rows": rows,
           "step_kernels": {"grid": [rn, rn, rn], "us_per_step": us, "alg_bytes_per_step": BYTES3_PER_NODE_STEP * rn ** 3,
                            "achieved_GBps": gbs, "peak_GBps": peak, "frac": gbs / peak, "peak_source": src,
                            "what": "two launches per step (k3_mprime, k3_phi)",
                            "one_launch": dict(kern[3], what="k3_step: one launch per step, m' recomputed on the "
                                                             "lower neighbours (36 B per voxel-step)")},
           "cpu_oracle": {"norm": 1, "s_per_solve": cpu_s, "solves_per_s": 1.0 / cpu_s, "cores": 1,
                          "w1_rel_diff_vs_gpu": abs(ref.w1 - rows[0]["w1_pair0"]) / abs(ref.w1),
                          "sample": "pair 0 replaying the GPU's per-level step counts"},
           "clocks": clk.summary()}
    print(json.dumps(out))
    return 0


SERVE_SIZES = (128, 256, 512, 1024)
SERVE_PROBS = (0.4, 0.3, 0.2, 0.1)


def serve_pool(torch, rank=0, per_size=(24, 16, 8, 4)):
    """Device-resident ellipse-texture pairs for each serving size."""
    import synth
    pool = {}
    for size, cnt in zip(SERVE_SIZES, per_size):
        pool[size] = []
        for k in range(cnt):
            r0, r1 = synth.pair(4, rank * 100000 + size * 100 + k, n=size)
            pool[size].append(tuple(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
                                    for x in (r0, r1)))
    return pool


def serve_run(w1, srv, pool, rate, n_req, seed, tol_of=None):
    """Poisson arrivals at `rate` req/s of mixed sizes and norms; returns
    (p50 ms, p99 ms, completed/s, statuses).  tol_of(n, norm): the request's
    eps_L (None: the library's default, eq. stop_tol)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_req)
    sizes = rng.choice(SERVE_SIZES, size=n_req, p=SERVE_PROBS)
    norms = rng.integers(1, 3, n_req)
    picks = rng.integers(0, 1 << 30, n_req)
    tickets = []
    t0 = time.perf_counter()
    t_next = t0
    for k in range(n_req):
        t_next += gaps[k]
        while True:
            d = t_next - time.perf_counter()
            if d <= 0:
                break
            time.sleep(min(d, 0.002))
        lst = pool[int(sizes[k])]
        a, b = lst[picks[k] % len(lst)]
        tol = tol_of(int(sizes[k]), int(norms[k])) if tol_of else 0.0
        tickets.append(srv.submit(a, b, norm=int(norms[k]), tol=tol))
    lat, statuses = [], []
    for k, t in enumerate(tickets):
        while True:
            st, v, stats, l = srv.poll(t)
            if st != w1.PENDING:
                break
            time.sleep(0.0005)
        statuses.append(st)
        if st != w1.OK and len(serve_run.failed) < 16:
            serve_run.failed.append({"size": int(sizes[k]), "norm": int(norms[k]), "status": int(st),
                                     "pair": int(picks[k] % len(pool[int(sizes[k])])),
                                     "iters": [int(x) for x in stats.iters] if stats else None,
                                     "fpr_over_tol": [f / t for f, t in zip(stats.fpr, stats.tol)] if stats else None})
        lat.append(l)
    t_end = time.perf_counter()
    lat = np.array(lat) * 1e3
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), n_req / (t_end - t0), statuses


serve_run.failed = []  # requests that ended with another status than W1_OK (first 16)


def serve_summary(w1, torch, args):
    """Short serving run for the default line: Poisson arrivals of the mixed
    sizes {128^2 .. 1024^2} at 0.4/0.3/0.2/0.1, both norms, 40 GB budget,
    requests at the benchmark's calibrated tolerance; one low rate and one
    high rate with at least 2000 requests."""
    pool = serve_pool(torch)
    out = []
    with w1.Server(hbm_budget_bytes=40 << 30, max_slots=args.slots, max_batch=args.serve_batch,
                   latency_below=args.latency_below, schedule=1) as srv:
        if args.latency_below > 0:
            for size in SERVE_SIZES:
                for norm in NORMS:
                    a0, a1 = pool[size][0]
                    srv.wait(srv.submit(a0, a1, norm=norm))
        serve_run(w1, srv, pool, 1000.0, 32, seed=1)
        for rate, n_req in ((float(r), int(q)) for r, q in (x.split(":") for x in args.serve_summary.split(","))):
            p50, p99, thr, sts = serve_run(w1, srv, pool, rate, n_req, seed=int(rate))
            out.append({"rate_req_s": rate, "requests": n_req, "p50_ms": p50, "p99_ms": p99, "solves_per_s": thr,
                        "not_ok": sum(1 for x in sts if x != w1.OK)})
        info = srv.info()
    return {"rates": out, "p50_ms": out[-1]["p50_ms"], "p99_ms": out[-1]["p99_ms"],
            "solves_per_s": out[-1]["solves_per_s"], "requests_at_headline_rate": out[-1]["requests"],
            "sizes": SERVE_SIZES, "probs": SERVE_PROBS, "budget_GiB": 40, "slots": args.slots,
            "latency_below": args.latency_below, "evictions": info.get("evictions"),
            "not_ok_requests": serve_run.failed,
            "what": "submit to completion (w1_poll_latency), Poisson arrivals; headline = the last rate"}


def mixed_summary(w1, torch, args):
    """The mixed-size batch (128 x 64^2 + 96 x 128^2 + 32 x 256^2, Gaussian
    mixtures, p = 2, the calibrated schedule unless --mixed-schedule 0) per
    pass: one persistent launch, per-size batched plans, and a loop of single
    solves; CUDA events on the launching stream, L2 flushed before each pass."""
    import synth
    stream = torch.cuda.current_stream()
    norm = args.mixed_norm
    passes = 1 + args.mixed_passes
    data = []
    for s in range(passes):
        per = []
        for ci, (n, B, _) in enumerate(MIXED):
            r = [synth.pair(3, 100000 * s + 1000 * ci + k, n=n) for k in range(B)]
            per.append(tuple(torch.from_numpy(np.ascontiguousarray(np.stack([x[j] for x in r]), dtype=np.float32)).cuda()
                             for j in (0, 1)))
        data.append(per)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    every = (w1.OK, w1.ERR_NOT_CONVERGED, w1.ERR_TIMEOUT, w1.ERR_MASS)
    total = sum(B for _, B, _ in MIXED)
    out, first = {}, None
    sch = args.mixed_schedule
    for mode in ("persistent", "lockstep", "loop"):
        if mode == "persistent":
            obj = w1.Mixed([(n, n, B) for n, B, _ in MIXED], norm=norm, schedule=sch)
        elif mode == "lockstep":
            obj = [w1.Plan(n, n, levels=L, norm=norm, batch=B, schedule=sch) for n, B, L in MIXED]
            lanes = [torch.cuda.Stream() for _ in MIXED]
        else:
            obj = [w1.Plan(n, n, levels=L, norm=norm, schedule=sch) for n, _, L in MIXED]

        def one_pass(s):
            flush.fill_(float(s))
            vals, sts = [], []
            if mode == "persistent":
                obj.solve_async([d[0] for d in data[s]], [d[1] for d in data[s]], stream=stream)
                stream.synchronize()
                for ci in range(len(MIXED)):
                    v, _, ps, _ = obj.results(ci, allow=every)
                    vals.extend(v)
                    sts.extend(ps)
            elif mode == "lockstep":
                ready = torch.cuda.Event()
                ready.record(stream)
                for ci in range(len(MIXED)):
                    lanes[ci].wait_event(ready)
                    obj[ci].solve_async(data[s][ci][0], data[s][ci][1], stream=lanes[ci])
                for ci in range(len(MIXED)):
                    stream.wait_stream(lanes[ci])
                    lanes[ci].synchronize()
                    v, _, ps, _ = obj[ci].results(allow=every)
                    vals.extend(v)
                    sts.extend(ps)
            else:
                for ci, (n, B, _) in enumerate(MIXED):
                    for b in range(B):
                        v, _, st_ = obj[ci].solve(data[s][ci][0][b], data[s][ci][1][b], stream=stream, allow=every)
                        vals.append(v)
                        sts.append(st_)
            return vals, sts

        one_pass(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [one_pass(s) for s in range(1, passes)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        vals = np.array([v for r in res for v in r[0]])
        n_ok = sum(1 for r in res for x in r[1] if x == w1.OK)
        if first is None:
            first = vals
        out[mode] = {"solves_per_s": n_ok / (ms / 1e3), "ms_per_pass": ms / (passes - 1),
                     "max_rel_diff_vs_persistent": float(np.max(np.abs(vals - first) / np.abs(first)))}
        if mode == "persistent":
            out[mode]["persistent_classes"] = [obj.persistent(c) for c in range(len(MIXED))]
            out[mode]["launch"] = obj.launch_info()
            obj.close()
        else:
            for p in obj:
                p.close()
    return {"workload": ", ".join(f"{B} x {n}^2 ({L} levels)" for n, B, L in MIXED), "norm": f"L{norm}",
            "schedule": "calibrated (w1_options.schedule = 1)" if sch else "the paper's (eq. stop_tol, alpha -1)",
            "pairs_per_pass": total, "passes": passes - 1, "modes": out,
            "speedup_vs_loop": out["persistent"]["solves_per_s"] / out["loop"]["solves_per_s"]}


def run_serve(args):
    import torch

    from paper_1810_00118_gb300 import w1

    pool = serve_pool(torch)
    rates = [float(x) for x in args.rates.split(",")]
    out = []
    with w1.Server(hbm_budget_bytes=40 << 30, max_slots=args.slots, max_batch=args.serve_batch,
                   latency_below=args.latency_below, schedule=1) as srv:
        # warm-up: requests one at a time build the latency-tuned slots (and run
        # the autotuner once per class), then a burst builds the others
        if args.latency_below > 0:
            for size in SERVE_SIZES:
                for norm in (1, 2):
                    a0, a1 = pool[size][0]
                    srv.wait(srv.submit(a0, a1, norm=norm))
        serve_run(w1, srv, pool, 1000.0, 16, seed=1)
        for r in rates:
            n = max(args.requests, int(r * args.min_seconds))
            p50, p99, thr, sts = serve_run(w1, srv, pool, r, n, seed=int(r))
            bad = sum(1 for x in sts if x not in (w1.OK, w1.ERR_NOT_CONVERGED))
            out.append({"rate_req_s": r, "requests": n, "p50_ms": p50, "p99_ms": p99, "solves_per_s": thr,
                        "failed": bad})
            print(json.dumps(out[-1]), flush=True)
        info = srv.info()
    print(json.dumps({"serving": out, "server": info, "sizes": SERVE_SIZES, "probs": SERVE_PROBS,
                      "budget_GiB": 40, "slots": args.slots, "max_batch": args.serve_batch,
                      "latency_below": args.latency_below}))
    return 0


def run_kernel_only(args):
    """One level's steps on an ellipse-texture density, timed with CUDA events."""
    import torch

    import synth
    from paper_1810_00118_gb300 import w1

    n = args.kn
    if args.only == "3d-kernel":
        # steps of the 3-D eq. primaldual (two launches each, or one with --kpath3 3) on an n^3 grid
        rng = np.random.default_rng(3)
        rho = torch.from_numpy(rng.normal(size=(n, n, n)).astype(np.float32)).cuda()
        rho -= rho.mean()
        st4 = [torch.zeros((n, n, n), device="cuda") for _ in range(4)]
        h = 1.0 / n
        mu = float(np.float32(0.5 * h / (2 * np.sqrt(3.0))))
        stream = torch.cuda.current_stream()
        kp = args.kpath3
        w1.cp_steps3d(rho, *st4, h, args.knorm, mu, mu, 4, path=kp, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = w1.cp_steps3d(rho, *st4, h, args.knorm, mu, mu, args.kiters, path=kp, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / args.kiters
        nb = BYTES3_PER_NODE_STEP if kp == 2 else BYTES3_ONE_LAUNCH
        print(json.dumps({"only": args.only, "n": n, "norm": args.knorm, "path": kp, "steps": args.kiters,
                          "us_per_step": us, "alg_GBps": nb * n ** 3 / (us * 1e-6) / 1e9, "fpr_last": r}))
        return 0
    r0, r1 = synth.pair(WORKLOAD, 0, n=n)
    rho = torch.from_numpy(np.ascontiguousarray(r0 - r1 - (r0 - r1).mean(), dtype=np.float32)).cuda()
    m1, m2, phi = (torch.zeros((n, n), device="cuda") for _ in range(3))
    h = 1.0 / n
    mu = float(np.float32(0.5 * h / (2 * np.sqrt(2.0))))
    stream = torch.cuda.current_stream()
    if args.only == "pdhg-kernel":
        # steps of eq. pdhg (Poisson solve by DCT) from zero on one level
        st = [torch.zeros((n, n), device="cuda") for _ in range(6)]
        w1.pdhg_steps(rho, *st, h, args.knorm, 4, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        G = w1.pdhg_steps(rho, *st, h, args.knorm, args.kiters, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"only": args.only, "n": n, "norm": args.knorm, "steps": args.kiters, "ms": ms,
                          "us_per_step": ms * 1e3 / args.kiters, "G_last": G}))
        return 0
    path = {"resident-kernel": 1, "stream-kernel": 2, "tblock-kernel": 3}[args.only]
    kw = {"cluster": args.kcluster} if path == 1 else {}
    w1.cp_steps(rho, m1, m2, phi, h, args.knorm, mu, mu, 4, path=path, stream=stream, **kw)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fpr = w1.cp_steps(rho, m1, m2, phi, h, args.knorm, mu, mu, args.kiters, path=path, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    us_step = ms * 1e3 / args.kiters
    print(json.dumps({"only": args.only, "n": n, "norm": args.knorm, "cluster": args.kcluster, "steps": args.kiters,
                      "ms": ms,
                      "us_per_step": us_step, "node_steps_per_s": n * n / (us_step * 1e-6),
                      "alg_GBps": 28.0 * n * n / (us_step * 1e-6) / 1e9, "fpr_last": fpr}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
