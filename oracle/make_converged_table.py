"""Writes tests/golden/converged_512.json: converged discrete W1 values of the
512 x 512 ellipse-texture pairs (synthetic workload 2, the benchmark's
workload) that the benchmark and the GPU tests compare against at relative
1e-4.  Calls only oracle/ (and the seeded input generators in synth/).

  - p = 1: the exact value of the discrete problem (eq. opt_flux_dis) by
    linear programming (oracle.exact, HiGHS with crossover).
  - p = 2: the FP64 oracle's Algorithm 3 with the eq. stop_tol schedule
    tightened 10^4 times (eps_L = 1e-6/128 * 1e-4); the value is the saddle
    value of eq. minmax_cp at the returned pair.  The same solve at 10^3 times
    is stored too: their difference bounds how far the stored value still is
    from the limit (it shrinks about threefold per factor ten).

Inputs are the FP32 densities the GPU receives (synth.to_f32_pair), balanced
by their FP64 mean.  Usage:
  python oracle/make_converged_table.py [--first 0] [--pairs 8] [--norms 1,2] [--workers N]
(rows are merged into an existing table).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

def _out(n, workload):
    name = "converged_512.json" if (n, workload) == (512, 2) else f"converged_w{workload}_{n}.json"
    return os.path.join(ROOT, "tests", "golden", name)


def _densities(workload, k, n):
    import synth
    r0, r1 = synth.pair(workload, k, n=n)
    _, _, d0, d1 = synth.to_f32_pair(r0, r1)
    return d0, d1


def _job(spec):
    norm, k, n, workload = spec
    import oracle
    from oracle import exact
    d0, d1 = _densities(workload, k, n)
    h = 1.0 / n
    levels = max(1, int(round(np.log2(n))) - 3)  # L = log2(1/h) - 3 (Sec. 5.3)
    t0 = time.time()
    if norm == 1:
        rho = d0 - d1
        rho = rho - rho.mean()
        return {"norm": 1, "pair": k, "w1": exact.w1_exact(rho, h, 1), "method": "LP", "seconds": time.time() - t0}
    eps_L = 1e-6 / 128 * (512.0 * h) ** 2  # eq. stop_tol
    a = oracle.multilevel(d0, d1, levels=levels, norm=norm, tol=eps_L * 1e-3, stop=oracle.STOP_FPR,
                          max_iters=20_000_000)
    b = oracle.multilevel(d0, d1, levels=levels, norm=norm, tol=eps_L * 1e-4, stop=oracle.STOP_FPR,
                          max_iters=20_000_000)
    return {"norm": norm, "pair": k, "w1": b.w1, "w1_at_1e-3": a.w1, "step": abs(b.w1 - a.w1) / b.w1,
            "iters": b.iters, "lb": b.stats.lb, "ub": b.stats.ub, "status": b.status,
            "method": "Algorithm 3, FP64, eps_L / 1e4, saddle value", "seconds": time.time() - t0}


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=8)
    ap.add_argument("--first", type=int, default=0, help="first pair index")
    ap.add_argument("--norms", default="1,2")
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--n", type=int, default=512, help="grid side")
    ap.add_argument("--workload", type=int, default=2, help="synth workload recipe")
    args = ap.parse_args()
    import oracle
    oracle.build()
    norms = [int(x) for x in args.norms.split(",")]
    specs = [(nm, k, args.n, args.workload) for nm in sorted(norms, reverse=True)
             for k in range(args.first, args.first + args.pairs)]
    with mp.get_context("spawn").Pool(args.workers) as pool:
        rows = pool.map(_job, specs, chunksize=1)
    out = _out(args.n, args.workload)
    table = {}
    if os.path.exists(out):
        with open(out) as f:
            table = json.load(f)
    table.update({
        "what": f"converged discrete W1 of {args.n}x{args.n} ellipse-texture pairs (synth workload {args.workload}, "
                f"seed {1000 * args.workload} + k), both ground norms; rho = rho0 - rho1 of the FP32 densities, "
                "balanced by its mean",
        "citation": "discrete problem eq. opt_flux_dis (Sec. 2.2); Algorithm 3 (Sec. 3.2); eq. stop_tol (Sec. 5.3); "
                    "saddle value = Lagrangian of eq. minmax_cp",
        "script": "oracle/make_converged_table.py",
        "grid": [args.n, args.n], "levels": max(1, int(round(np.log2(args.n))) - 3), "workload": args.workload})
    for r in rows:
        table.setdefault(f"L{r['norm']}", {})[str(r["pair"])] = r
    with open(out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(f"wrote {out}")


if __name__ == "__main__":
    main()
