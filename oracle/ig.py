"""Iterated greedy heuristic (Ruiz and Stuetzle 2007) for an initial upper
bound of the permutation flow-shop.  Not part of the paper's method: the
tests use it only to start the oracle's branch-and-bound from a tighter
incumbent than NEH gives.  The optimum the B&B reports does not depend on
where it starts, as long as the start is the makespan of a real schedule,
which the returned value always is (it is recomputed from the returned
sequence).  TEST INFRASTRUCTURE ONLY.

Steps (Ruiz and Stuetzle, "A simple and effective iterated greedy algorithm
for the permutation flowshop scheduling problem", EJOR 177, 2007):
  - start from the NEH sequence;
  - destruction: remove `d` jobs chosen at random;
  - construction: reinsert them one by one, each at the position that
    minimises the partial makespan (first such position on ties);
  - acceptance: keep the new sequence if it is no worse, else keep it with
    probability exp(-(new - cur) / T), T = tau * sum(p) / (10 n m);
  - remember the best sequence seen.
"""
import math
import random

from oracle.brute import makespan
from oracle.neh import neh


def _insert_best(p, seq, j):
    best = None
    for pos in range(len(seq) + 1):
        cand = seq[:pos] + [j] + seq[pos:]
        v = makespan(p, cand)
        if best is None or v < best[0]:
            best = (v, cand)
    return best


def iterated_greedy(p, iterations=2000, d=4, tau=0.4, seed=0):
    """Returns (makespan, sequence) of the best schedule found."""
    n, m = len(p), len(p[0])
    rng = random.Random(seed)
    cur_v, cur = neh(p)
    best_v, best = cur_v, list(cur)
    if n <= 1:
        return best_v, best
    temp = tau * sum(int(x) for row in p for x in row) / (10.0 * n * m)
    d = min(d, n - 1)
    for _ in range(iterations):
        seq = list(cur)
        removed = []
        for _ in range(d):
            removed.append(seq.pop(rng.randrange(len(seq))))
        v = None
        for j in removed:
            v, seq = _insert_best(p, seq, j)
        if v <= cur_v:
            cur_v, cur = v, seq
            if v < best_v:
                best_v, best = v, list(seq)
        elif rng.random() < math.exp(-(v - cur_v) / temp):
            cur_v, cur = v, seq
    return makespan(p, best), best
