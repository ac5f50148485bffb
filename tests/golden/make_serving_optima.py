"""Writes tests/golden/serving_optima.json: the optimum of each of the 32
serving-loop searches (20 jobs, m=5 for seeds 200-215, m=10 for 216-231),
found by the CPU oracle's branch-and-bound.  Calls only oracle/ (plus the
seeded input generator).

Method per seed:
  - ub0 = the best of the oracle's NEH schedule and three seeded runs of its
    iterated greedy heuristic (each value is the makespan of a real
    schedule, so ub0 >= the optimum and the search cannot miss it);
  - the tree is cut at depth 2: one oracle search per ordered pair of first
    jobs (n (n - 1) subtrees), every node bounded with the per-job release
    times, each asked for a schedule of makespan <= ub0 - 1 (the schedule
    behind ub0 is the incumbent, so nodes whose bound reaches ub0 are cut
    at once); the subtrees of all depth-2 prefixes cover every schedule, so
    the smallest subtree optimum is the instance's optimum, and when no
    subtree finds one the optimum is ub0 itself;
  - the subtree searches of all seeds share one process pool, so a hard seed
    uses every core.
A seed whose searches do not all finish within the time limit keeps its
earlier entry (or null: unverified).

    python tests/golden/make_serving_optima.py [seconds] [workers] [seed ...]
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serving_optima.json")
IG_ITERATIONS = 6000
IG_RUNS = 3


def upper_bound(args):
    seed, p, run = args
    from oracle.ig import iterated_greedy
    v, seq = iterated_greedy(p, iterations=IG_ITERATIONS, seed=run)
    return seed, v, seq


def subtree(args):
    seed, p, ub0, prefix = args
    import oracle
    t0 = time.time()
    rc, best, perm, nodes = oracle.branch_and_bound(p, ub0 - 1, oracle.RELEASE_EST, prefix)
    return seed, rc == oracle.FO_OK, best, perm.tolist(), nodes, time.time() - t0


def main():
    limit = float(sys.argv[1]) if len(sys.argv) > 1 else 3600.0
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count() or 1
    only = {int(s) for s in sys.argv[3:]}
    from paper_1208_3933_gb300 import workloads
    import oracle
    from oracle.neh import neh
    from oracle.brute import makespan
    oracle.build()
    jobs = [(s, p) for s, p in workloads.serving_searches() if not only or s in only]
    results = {}
    if os.path.exists(OUT):
        results = json.load(open(OUT))["results"]
    for s, p in workloads.serving_searches():
        results.setdefault(str(s), {"m": int(p.shape[1]), "opt": None})

    def save():
        json.dump({"what": "optima of the serving-loop searches from the CPU oracle's branch-and-bound",
                   "results": results}, open(OUT, "w"), indent=1)

    t_end = time.time() + limit
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        ub = {}
        for s, p in jobs:
            v, seq = neh(p)
            ub[s] = (v, "neh", list(seq))
        for seed, v, seq in pool.imap_unordered(
                upper_bound, [(s, p, r) for s, p in jobs for r in range(IG_RUNS)]):
            p = dict(jobs)[seed]
            assert v == makespan(p, seq) and sorted(seq) == list(range(p.shape[0]))
            if v < ub[seed][0]:
                ub[seed] = (v, "iterated greedy", list(seq))
        tasks = []
        for s, p in jobs:
            n = p.shape[0]
            tasks += [(s, p, ub[s][0], (a, b)) for a in range(n) for b in range(n) if a != b]
        left = {s: 0 for s, _ in jobs}
        for t in tasks:
            left[t[0]] += 1
        acc = {s: {"best": None, "perm": None, "nodes": 0, "seconds": 0.0} for s, _ in jobs}
        it = pool.imap_unordered(subtree, tasks)
        while any(left.values()):
            try:
                seed, ok, best, perm, nodes, secs = it.next(timeout=max(1.0, t_end - time.time()))
            except mp.TimeoutError:
                break
            a = acc[seed]
            a["nodes"] += nodes
            a["seconds"] += secs
            if ok and (a["best"] is None or best < a["best"]):
                a["best"], a["perm"] = best, perm
            left[seed] -= 1
            if left[seed] == 0:
                p = dict(jobs)[seed]
                if a["best"] is None:  # no schedule below ub0: the ub0 schedule is optimal
                    a["best"], a["perm"] = ub[seed][0], ub[seed][2]
                assert a["best"] == makespan(p, a["perm"]) and a["best"] <= ub[seed][0]
                results[str(seed)] = {"m": int(p.shape[1]), "ub0": ub[seed][0], "ub0_from": ub[seed][1],
                                      "opt": a["best"], "perm": a["perm"], "oracle_nodes": a["nodes"],
                                      "cpu_seconds": round(a["seconds"], 1),
                                      "method": "depth-2 subtrees, per-job release times"}
                save()
                print(seed, results[str(seed)]["opt"], a["nodes"], round(a["seconds"]), flush=True)
        pool.terminate()
    save()


if __name__ == "__main__":
    main()
