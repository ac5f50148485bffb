"""CPU oracle for the permutation flow-shop two-machine lower bound.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is shared
with, or called by, the CUDA library in ``paper_1208_3933_gb300``.

The arithmetic lives in ``fsp_oracle.c`` (plain C, int64, single-threaded);
this module compiles it with gcc on first use and wraps it with ctypes.
``oracle.brute`` holds the brute-force enumerations that pin it.

Paper: Melab et al., "A GPU-accelerated Branch-and-Bound Algorithm for the
Flow-Shop Scheduling Problem", Sections II-B..II-D and the LB pseudo-code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsp_oracle.c")
_LIB = os.path.join(_HERE, "_fsp_oracle.so")
_lock = threading.Lock()
_lib = None

FO_OK = 0
FO_EINVAL = -1
FO_ENOMEM = -2
FO_EBADNODE = -4
FO_ENOTFOUND = -6
RELEASE_HEADS = 0  # release of k: max(C(sigma,k), min_U sum_{h<k} p_jh)
RELEASE_EST = 1    # release of k: min_U earliest start of j on k after the prefix


def build(force: bool = False) -> str:
    """Compiles fsp_oracle.c into _fsp_oracle.so (plain -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i16p = ctypes.POINTER(ctypes.c_int16)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.fo_num_pairs.argtypes = [ctypes.c_int]
            lib.fo_num_pairs.restype = ctypes.c_int
            lib.fo_tables.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p]
            lib.fo_tables.restype = ctypes.c_int
            lib.fo_lb.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, i16p,
                                  ctypes.c_int32, i64p, i32p]
            lib.fo_lb.restype = ctypes.c_int
            lib.fo_lb_pool.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, i16p,
                                       i32p, ctypes.c_int64, i32p]
            lib.fo_lb_pool.restype = ctypes.c_int64
            lib.fo_lb_ex.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, i16p,
                                     ctypes.c_int32, ctypes.c_int, i64p, i32p]
            lib.fo_lb_ex.restype = ctypes.c_int
            lib.fo_lb_pool_ex.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, i16p,
                                          i32p, ctypes.c_int64, ctypes.c_int, i32p]
            lib.fo_lb_pool_ex.restype = ctypes.c_int64
            lib.fo_bnb.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32, i16p, i32p, i64p]
            lib.fo_bnb.restype = ctypes.c_int
            lib.fo_bnb_ex.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32, ctypes.c_int, i16p,
                                      ctypes.c_int32, i16p, i32p, i64p]
            lib.fo_bnb_ex.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Tables:
    """The per-instance tables of Section II-D as the oracle builds them:
    ``mm`` [P,2] couples (k<l, lexicographic), ``lag`` [P,n], ``jm`` [P,n]."""

    def __init__(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.int32)
        if p.ndim != 2 or p.shape[0] < 1 or p.shape[1] < 2:
            raise ValueError("p must be [n][m] with n>=1, m>=2")
        self.p = p
        self.n, self.m = p.shape
        lib = _load()
        self.P = lib.fo_num_pairs(self.m)
        self.mm = np.zeros((self.P, 2), np.int32)
        self.lag = np.zeros((self.P, self.n), np.int32)
        self.jm = np.zeros((self.P, self.n), np.int32)
        rc = lib.fo_tables(self.n, self.m, _ptr(p, ctypes.c_int32), _ptr(self.mm, ctypes.c_int32),
                           _ptr(self.lag, ctypes.c_int32), _ptr(self.jm, ctypes.c_int32))
        if rc != FO_OK:
            raise RuntimeError(f"fo_tables failed: {rc}")

    def lb(self, prefix, return_pairs: bool = False, release: int = 0):
        """LB of the node whose scheduled prefix is ``prefix`` (a sequence of
        job indices).  Returns None for an invalid prefix.  ``release`` picks
        the reading of RM: RELEASE_HEADS (default) or RELEASE_EST."""
        lib = _load()
        row = np.zeros(self.n, np.int16)
        d = len(prefix)
        if d > self.n:
            return None
        row[:d] = np.asarray(prefix, dtype=np.int16)
        pairs = np.zeros(self.P, np.int64)
        out = ctypes.c_int32(0)
        rc = lib.fo_lb_ex(self.n, self.m, _ptr(self.p, ctypes.c_int32), _ptr(self.mm, ctypes.c_int32),
                          _ptr(self.lag, ctypes.c_int32), _ptr(self.jm, ctypes.c_int32),
                          _ptr(row, ctypes.c_int16), d, int(release), _ptr(pairs, ctypes.c_int64),
                          ctypes.byref(out))
        if rc == FO_EBADNODE:
            return None
        if rc != FO_OK:
            raise RuntimeError(f"fo_lb failed: {rc}")
        return (int(out.value), pairs) if return_pairs else int(out.value)

    def lb_pool(self, rows: np.ndarray, depths: np.ndarray, threads: int = 1, release: int = 0) -> np.ndarray:
        """Bounds a pool (rows int16 [N][n], depths int32 [N]); invalid rows
        give -1.  ``threads`` > 1 runs the single-threaded C routine on
        disjoint chunks from a thread pool (ctypes drops the GIL)."""
        lib = _load()
        rows = np.ascontiguousarray(rows, dtype=np.int16)
        depths = np.ascontiguousarray(depths, dtype=np.int32)
        N = depths.shape[0]
        if rows.shape != (N, self.n):
            raise ValueError("rows must be [N][n]")
        out = np.empty(N, np.int32)
        if N == 0:
            return out

        def run(lo, hi):
            rc = lib.fo_lb_pool_ex(self.n, self.m, _ptr(self.p, ctypes.c_int32),
                                   _ptr(self.mm, ctypes.c_int32), _ptr(self.lag, ctypes.c_int32),
                                   _ptr(self.jm, ctypes.c_int32),
                                   _ptr(rows[lo:hi], ctypes.c_int16), _ptr(depths[lo:hi], ctypes.c_int32),
                                   hi - lo, int(release), _ptr(out[lo:hi], ctypes.c_int32))
            if rc < 0:
                raise RuntimeError(f"fo_lb_pool failed: {rc}")

        threads = max(1, min(int(threads), N))
        if threads == 1:
            run(0, N)
        else:
            bounds = np.linspace(0, N, threads + 1).astype(np.int64)
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda t: run(int(bounds[t]), int(bounds[t + 1])), range(threads)))
        return out


def branch_and_bound(p: np.ndarray, ub0: int, release: int = RELEASE_HEADS, prefix=()):
    """Depth-first B&B of fsp_oracle.c, every node bounded with the given
    reading of RM, over the subtree of ``prefix`` (the whole tree when it is
    empty).  Returns (status, best_makespan, best_perm, nodes_bounded);
    status is FO_OK or FO_ENOTFOUND."""
    lib = _load()
    p = np.ascontiguousarray(p, dtype=np.int32)
    n, m = p.shape
    perm = np.zeros(n, np.int16)
    root = np.zeros(max(1, len(prefix)), np.int16)
    root[:len(prefix)] = np.asarray(prefix, dtype=np.int16)
    best = ctypes.c_int32(0)
    nodes = ctypes.c_int64(0)
    rc = lib.fo_bnb_ex(n, m, _ptr(p, ctypes.c_int32), int(ub0), int(release), _ptr(root, ctypes.c_int16),
                       len(prefix), _ptr(perm, ctypes.c_int16), ctypes.byref(best), ctypes.byref(nodes))
    if rc == FO_EBADNODE:
        raise ValueError(f"invalid prefix {list(prefix)}")
    if rc not in (FO_OK, FO_ENOTFOUND):
        raise RuntimeError(f"fo_bnb failed: {rc}")
    return rc, int(best.value), perm, int(nodes.value)
