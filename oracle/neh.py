"""NEH constructive heuristic (Nawaz, Enscore, Ham 1983) for an initial upper
bound of the permutation flow-shop.  Not part of the paper's method: the
tests use it only to start the oracle's branch-and-bound from a good
incumbent.  TEST INFRASTRUCTURE ONLY."""
from oracle.brute import makespan


def neh(p):
    """Jobs by decreasing total processing time, each inserted at the
    position that minimises the partial makespan (first such position on
    ties).  Returns (makespan, sequence)."""
    n = len(p)
    order = sorted(range(n), key=lambda j: (-int(sum(int(x) for x in p[j])), j))
    seq = [order[0]]
    for j in order[1:]:
        best = None
        for pos in range(len(seq) + 1):
            cand = seq[:pos] + [j] + seq[pos:]
            v = makespan(p, cand)
            if best is None or v < best[0]:
                best = (v, cand)
        seq = best[1]
    return makespan(p, seq), seq
