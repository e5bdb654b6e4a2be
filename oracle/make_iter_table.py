"""Writes oracle/iter_table.json: the oracle's own per-level iteration counts
(Algorithm 3, eq. stop_tol tolerances, alpha = -1, K = 32) on the 512x512
ellipse-texture pairs 0..3, for both norms.  Used to scale the CPU-baseline
timing; calls only the oracle and the input generators."""
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def run(job):
    import oracle
    import synth
    norm, k = job
    r0, r1 = synth.pair(2, k)
    _, _, d0, d1 = synth.to_f32_pair(r0, r1)
    h = 1.0 / 512
    eps = 1e-6 / 128 * (512 * h) ** 2
    res = oracle.multilevel(d0, d1, levels=6, norm=norm, tol=eps, alpha=-1.0, stop=oracle.STOP_FPR, check_every=32)
    return norm, k, res.iters, res.w1


if __name__ == "__main__":
    import multiprocessing as mp
    import oracle
    oracle.build()
    jobs = [(n, k) for n in (1, 2) for k in range(4)]
    table = {"1": {}, "2": {}, "w1": {"1": {}, "2": {}}}
    with ProcessPoolExecutor(max_workers=8, mp_context=mp.get_context("spawn")) as ex:
        for norm, k, iters, w1 in ex.map(run, jobs):
            table[str(norm)][str(k)] = iters
            table["w1"][str(norm)][str(k)] = w1
            print(norm, k, iters, w1, flush=True)
    with open(os.path.join(HERE, "iter_table.json"), "w") as f:
        json.dump(table, f, indent=1)
