"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no bounding arithmetic: it only draws processing times and
node pools, and both the CUDA path and the CPU oracle are fed from it.

Recipe (every draw comes from ``numpy.random.default_rng(seed)``):
  * processing times ``p`` [n][m] int32, uniform on 1..99 (the range of
    Taillard's flow-shop instances, which the paper measures on; the instances
    themselves are not used), drawn first;
  * a pool of N nodes drawn next from the same stream: every row is an
    independent random permutation of 0..n-1 stored as int16 (only its first
    ``depth`` entries are the scheduled prefix), and ``depth`` is uniform on
    0..n-1 (int32).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def processing_times(rng: np.random.Generator, n: int, m: int) -> np.ndarray:
    return rng.integers(1, 100, size=(n, m), dtype=np.int32)


def random_pool(rng: np.random.Generator, n: int, N: int, max_depth: int | None = None):
    """N random prefixes: rows int16 [N][n] (random permutations), depths
    int32 [N] uniform on 0..max_depth-1 (default 0..n-1)."""
    if max_depth is None:
        max_depth = n
    rows = rng.permuted(np.tile(np.arange(n, dtype=np.int16), (N, 1)), axis=1)
    depths = rng.integers(0, max_depth, N, dtype=np.int32)
    return np.ascontiguousarray(rows), depths


@dataclass
class PoolWorkload:
    name: str
    n: int
    m: int
    seed: int
    p: np.ndarray
    rows: np.ndarray
    depths: np.ndarray

    @property
    def N(self) -> int:
        return int(self.depths.shape[0])


def pool_workload(name: str, n: int, m: int, seed: int, N: int) -> PoolWorkload:
    rng = np.random.default_rng(seed)
    p = processing_times(rng, n, m)
    rows, depths = random_pool(rng, n, N)
    return PoolWorkload(name, n, m, seed, p, rows, depths)


# The bounding-pool workloads: 20x20 (seed 1, 65,536 nodes), 200x20
# (seed 2, 262,144 nodes) and 500x20 (seed 2, 65,536 nodes, forces pair-tiled
# staging of the tables).
POOL_CONFIGS = {
    "pool_20x20": dict(n=20, m=20, seed=1, N=65536),
    "pool_200x20": dict(n=200, m=20, seed=2, N=262144),
    "pool_500x20": dict(n=500, m=20, seed=2, N=65536),
}


def named_pool(name: str, N: int | None = None) -> PoolWorkload:
    cfg = dict(POOL_CONFIGS[name])
    if N is not None:
        cfg["N"] = N
    return pool_workload(name, **cfg)


def small_bnb_instance(seed: int = 0, n: int = 8, m: int = 5) -> np.ndarray:
    """The plain-method instance: n=8 jobs x m=5 machines, seed 0."""
    return processing_times(np.random.default_rng(seed), n, m)


def trivial_ub(p: np.ndarray) -> int:
    """Sum of machine-1 times plus the largest tail (sum over machines 2..m)
    of any job: the upper-bound formula quoted for the plain-method instance.
    It is not a valid upper bound in general (for n=2, m=2 and both jobs
    (1,10) it gives 12 against an optimum of 21), so callers combine it with
    the makespan of a complete schedule."""
    return int(p[:, 0].sum() + (p[:, 1:].sum(axis=1)).max())


def batched_instances(seeds=range(100, 164)):
    """64 instances of the batched uneven launch: from each seed's stream,
    n from {20,50,100,200}, m from {5,10,20}, then p, then the pool size
    N = round(exp(U(ln 1024, ln 65536))), then the pool."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        n = int(rng.choice([20, 50, 100, 200]))
        m = int(rng.choice([5, 10, 20]))
        p = processing_times(rng, n, m)
        N = int(round(math.exp(rng.uniform(math.log(1024), math.log(65536)))))
        rows, depths = random_pool(rng, n, N)
        out.append(PoolWorkload(f"batch_seed{s}", n, m, s, p, rows, depths))
    return out


def serving_searches(seeds=range(200, 232)):
    """The 32 DFS searches of the serving loop: n=20, m=5 for seeds 200-215
    and m=10 for seeds 216-231."""
    out = []
    for s in seeds:
        m = 5 if s < 216 else 10
        out.append((s, processing_times(np.random.default_rng(s), 20, m)))
    return out


def serving_streams(n_streams: int = 16, seed: int = 300, pools_per_stream: int = 8,
                    rate_hz: float = 200.0):
    """Synthetic 200x20 pool streams: per stream a fixed instance (seed+i), and
    pools of log-uniform size 4,096..32,768 arriving as a Poisson process of
    the given rate.  Returns a list of (instance p, [(t_arrival_s, rows,
    depths), ...])."""
    out = []
    for i in range(n_streams):
        rng = np.random.default_rng(seed + i)
        p = processing_times(rng, 200, 20)
        t = 0.0
        pools = []
        for _ in range(pools_per_stream):
            t += float(rng.exponential(1.0 / rate_hz))
            N = int(round(math.exp(rng.uniform(math.log(4096), math.log(32768)))))
            rows, depths = random_pool(rng, 200, N)
            pools.append((t, rows, depths))
        out.append((p, pools))
    return out
