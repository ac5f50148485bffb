"""Writes tests/golden/serving_optima.json: the optimum of each of the 32
serving-loop searches (20 jobs, m=5 for seeds 200-215, m=10 for 216-231),
found by the CPU oracle's branch-and-bound started from the oracle's NEH
schedule.  Calls only oracle/ (plus the seeded input generator).  Searches
that do not finish within the per-seed time limit are stored as null.

    python tests/golden/make_serving_optima.py [seconds_per_seed] [workers]
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def solve(args):
    seed, p = args
    import oracle
    from oracle.neh import neh
    ub, _ = neh(p)
    t0 = time.time()
    rc, best, perm, nodes = oracle.branch_and_bound(p, ub)
    return seed, int(p.shape[1]), ub, rc, best, perm.tolist(), nodes, time.time() - t0


def main():
    limit = float(sys.argv[1]) if len(sys.argv) > 1 else 600.0
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count() or 1
    from paper_1208_3933_gb300 import workloads
    import oracle
    oracle.build()
    jobs = workloads.serving_searches()
    out_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serving_optima.json")
    results = {str(s): {"m": int(p.shape[1]), "opt": None} for s, p in jobs}
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers)
    pending = {s: pool.apply_async(solve, ((s, p),)) for s, p in jobs}
    t_end = time.time() + limit
    for s, fut in pending.items():
        try:
            seed, m, ub, rc, best, perm, nodes, secs = fut.get(timeout=max(1.0, t_end - time.time()))
        except mp.TimeoutError:
            continue
        results[str(seed)] = {"m": m, "neh": ub, "opt": best if rc == oracle.FO_OK else None,
                              "perm": perm, "oracle_nodes": nodes, "seconds": round(secs, 2)}
        json.dump({"what": "optima of the serving-loop searches from the CPU oracle (NEH start)",
                   "results": results}, open(out_path, "w"), indent=1)
    pool.terminate()
    json.dump({"what": "optima of the serving-loop searches from the CPU oracle (NEH start)",
               "results": results}, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main()
