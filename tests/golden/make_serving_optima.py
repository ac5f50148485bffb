"""Writes tests/golden/serving_optima.json: the optimum of each of the 32
serving-loop searches (20 jobs, m=5 for seeds 200-215, m=10 for 216-231),
found by the CPU oracle's branch-and-bound.  Calls only oracle/ (plus the
seeded input generator).

Method per seed:
  - the incumbent starts as the best of the oracle's NEH schedule and three
    seeded runs of its iterated greedy heuristic (real schedules, so the
    incumbent's makespan is never below the optimum);
  - the tree is cut at depth 2: one oracle search per ordered pair of first
    jobs (n (n - 1) subtrees, taken in increasing order of their root bound),
    every node bounded with the per-job release times;
  - each subtree search is started with the incumbent known at that moment,
    U, and asked for a schedule of makespan <= U - 1 (nodes whose bound
    reaches U are cut at once); a schedule it finds becomes the incumbent
    for the subtrees started later;
  - the subtrees of all depth-2 prefixes cover every schedule, so when all
    are done the incumbent is optimal: a better schedule would lie in some
    subtree, whose search was started with an incumbent above it and so
    would have returned it.
The subtree searches of all seeds share one process pool (seeds in the order
given), so a hard seed uses every core.  A seed whose searches do not all
finish within the time limit keeps its earlier entry (or null: unverified).
With --checkpoint FILE, finished subtrees are recorded there and a restart
skips them.

    python tests/golden/make_serving_optima.py [--checkpoint FILE] [seconds] [workers] [seed ...]
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
    seed, p, ub, prefix = args
    import oracle
    t0 = time.time()
    rc, best, perm, nodes = oracle.branch_and_bound(p, ub - 1, oracle.RELEASE_EST, prefix)
    return seed, prefix, ub, rc == oracle.FO_OK, best, perm.tolist(), nodes, time.time() - t0


def main():
    argv = sys.argv[1:]
    ckpt_path = None
    if argv[:1] == ["--checkpoint"]:
        ckpt_path, argv = argv[1], argv[2:]
    limit = float(argv[0]) if len(argv) > 0 else 3600.0
    workers = int(argv[1]) if len(argv) > 1 else os.cpu_count() or 1
    order = [int(s) for s in argv[2:]]
    from paper_1208_3933_gb300 import workloads
    import oracle
    from oracle.neh import neh
    from oracle.brute import makespan
    oracle.build()
    probs = dict(workloads.serving_searches())
    order = order or sorted(probs)
    results = json.load(open(OUT))["results"] if os.path.exists(OUT) else {}
    for s, p in probs.items():
        results.setdefault(str(s), {"m": int(p.shape[1]), "opt": None})
    ckpt = json.load(open(ckpt_path)) if ckpt_path and os.path.exists(ckpt_path) else {}

    def save():
        json.dump({"what": "optima of the serving-loop searches from the CPU oracle's branch-and-bound",
                   "results": results}, open(OUT, "w"), indent=1)

    t_end = time.time() + limit
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        inc = {}  # seed -> (makespan, sequence, where from)
        for s in order:
            v, seq = neh(probs[s])
            inc[s] = (v, list(seq), "neh")
        for seed, v, seq in pool.imap_unordered(upper_bound,
                                                [(s, probs[s], r) for s in order for r in range(IG_RUNS)]):
            assert v == makespan(probs[seed], seq) and sorted(seq) == list(range(probs[seed].shape[0]))
            if v < inc[seed][0]:
                inc[seed] = (v, list(seq), "iterated greedy")
        start = {s: inc[s] for s in order}
        acc = {s: {"nodes": 0, "seconds": 0.0, "left": 0} for s in order}
        queue = []
        for s in order:
            p, n = probs[s], probs[s].shape[0]
            t = oracle.Tables(p)
            prefixes = [(a, b) for a in range(n) for b in range(n) if a != b]
            done = ckpt.get(str(s), {})
            for pre in prefixes:
                rec = done.get(f"{pre[0]},{pre[1]}")
                if rec:  # restart: a subtree finished earlier
                    acc[s]["nodes"] += rec["nodes"]
                    acc[s]["seconds"] += rec["seconds"]
                    if rec["best"] is not None and rec["best"] < inc[s][0]:
                        inc[s] = (rec["best"], rec["perm"], "subtree search")
            todo = [pre for pre in prefixes if f"{pre[0]},{pre[1]}" not in done]
            todo.sort(key=lambda pre: (t.lb(list(pre), release=oracle.RELEASE_EST), pre))
            acc[s]["left"] = len(todo)
            queue += [(s, pre) for pre in todo]

        def finish(s):
            p = probs[s]
            best, perm, how = inc[s]
            assert best == makespan(p, perm) and sorted(perm) == list(range(p.shape[0]))
            results[str(s)] = {"m": int(p.shape[1]), "neh": neh(p)[0], "start": start[s][0],
                               "start_from": start[s][2], "opt": best, "perm": list(map(int, perm)),
                               "oracle_nodes": acc[s]["nodes"], "cpu_seconds": round(acc[s]["seconds"], 1),
                               "method": "depth-2 subtrees, per-job release times, shared incumbent"}
            save()
            print(s, best, acc[s]["nodes"], round(acc[s]["seconds"]), flush=True)

        for s in order:
            if acc[s]["left"] == 0:
                finish(s)
        pending = []
        qi = 0
        while pending or qi < len(queue):
            while qi < len(queue) and len(pending) < workers:
                s, pre = queue[qi]
                qi += 1
                pending.append(pool.apply_async(subtree, ((s, probs[s], inc[s][0], pre),)))
            if time.time() > t_end:
                break
            ready = [f for f in pending if f.ready()]
            if not ready:
                time.sleep(0.05)
                continue
            for f in ready:
                pending.remove(f)
                seed, pre, ub, ok, best, perm, nodes, secs = f.get()
                a = acc[seed]
                a["nodes"] += nodes
                a["seconds"] += secs
                a["left"] -= 1
                if ok and best < inc[seed][0]:
                    inc[seed] = (best, perm, "subtree search")
                if ckpt_path:
                    ckpt.setdefault(str(seed), {})[f"{pre[0]},{pre[1]}"] = {
                        "ub": ub, "best": best if ok else None, "perm": perm if ok else None,
                        "nodes": nodes, "seconds": round(secs, 2)}
                    json.dump(ckpt, open(ckpt_path, "w"))
                if a["left"] == 0:
                    finish(seed)
        pool.terminate()
    save()


if __name__ == "__main__":
    main()
