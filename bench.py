#!/usr/bin/env python3
"""Benchmark: lower-bound evaluations per second at n x m = 200 x 20.

One step bounds the whole 200x20 pool (262,144 random-prefix nodes, seed 2)
with fsp_bound_pool: every node's prefix recurrence, release/latency minima
and the filtered Johnson scan of all 190 machine couples, i.e. one full pass
of the bounding operator.  Inputs are resident in HBM before the timed region;
three copies of the pool (3 x 105 MB > the 129 MB L2) are used in rotation so
no step finds its input in L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank bounds its own pool
of the same size (weak scaling, no collective on the data path; the ranks
meet only in the barriers and the max-over-ranks of the timing).
``--impl reference`` times the CPU oracle (the plain C bounder, all host
cores) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "pool_200x20"
METRIC = "LB evals/s at n×m=200×20"
UNIT = "nodes/s"


def algorithmic_int_ops(n: int, m: int, depths: np.ndarray) -> float:
    """Integer operations of the bound per the method's own cost model:
    per couple one membership test for each of the n Johnson entries and four
    updates (add, add, max, add) for each of the n' = n - d unscheduled ones;
    per node 2mn for the release/latency minima and 2md for the prefix
    recurrence.  Summed over the nodes of one launch."""
    P = m * (m - 1) // 2
    d = depths.astype(np.float64)
    nu = n - d
    return float(np.sum(P * (n + 4 * nu) + 2 * m * n + 2 * m * d))


LANES_SOURCES = ("fsp_bound_lanes.cu", "fsp_bound_streamed28.cu", "fsp_bound_global.cu", "fsp_bound_resident.cu",
                 "fsp_lanes_device.cuh",
                 "fsp_batch_scan.cuh", "fsp_plan.h", "fsp_internal.h", "fsp_ptx.cuh", "fsp_instance.cpp")


def kernel_source_hash() -> str:
    """Hash of the sources that make up the couple-lanes bounding kernel."""
    h = hashlib.sha256()
    for name in LANES_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1208_3933_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def kernel_name(cfg) -> str:
    """The dominant kernel of a launch shape (its name in ncu launch lists)."""
    if not cfg or cfg.get("kernel") == 1:
        return "fsp_bound_kernel (node-lockstep)"
    if cfg.get("staging") == 2 and cfg.get("nodes_per_thread") in (28, 56):
        return "fsp_lanes_streamed28"
    return {1: "fsp_lanes_resident", 2: "fsp_lanes_streamed", 3: "fsp_lanes_scan (after fsp_lanes_prep)",
            4: "fsp_lanes_warp", 5: "fsp_lanes_global"}.get(cfg.get("staging"), "fsp_lanes_streamed")


def read_traffic(n_nodes: int):
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on the current kernel sources (else None).  The capture is a smaller pool
    of the same instance; the bytes per node are scaled to this launch's nodes
    (the kernel reads each node's row once and writes one bound)."""
    path = os.path.join(ROOT, "profiles", "fsp_lanes_streamed_pool_200x20.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d["dram_bytes_per_launch"] / d["nodes_per_launch"] * n_nodes


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def alu_peak_ops(sm_count: int, sm_max_mhz: float, lanes_per_sm: int) -> float:
    return sm_count * lanes_per_sm * sm_max_mhz * 1e6


# Integer operations per SM per clock behind the roofline: the add+max
# pattern of the bound issues one add and one max per lane per clock on the
# two integer-capable pipes (64 lanes each); the probe in
# paper_1208_3933_gb300/microbench/alu_peak.cu measures 127 of 128
# (python bench.py --alu-peak).
ALU_LANES_PER_SM = 128


def run_alu_peak():
    import ctypes

    import torch
    from paper_1208_3933_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.MICRO_LIB)
    f = lib.fsp_microbench_alu
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_float)] * 2 + [ctypes.POINTER(ctypes.c_double)]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    names = ["add+max (the bound's recurrence)", "logic (one lop3 per step)", "imad", "fadd+fmax"]
    for pat, name in zip([0, 2, 3, 4], names):
        ms, mhz, ops = ctypes.c_float(), ctypes.c_float(), ctypes.c_double()
        blocks = sms * 8
        rc = f(pat, blocks, 2000, ctypes.byref(ms), ctypes.byref(mhz), ctypes.byref(ops))
        total = ops.value * blocks * 256
        if pat == 2:
            total /= 2  # the compiler fuses the three logic ops into one lop3
        rate = total / (ms.value * 1e-3)
        print(json.dumps({"pattern": name, "rc": rc, "ms": round(ms.value, 4), "sm_mhz": round(mhz.value),
                          "int_ops_per_s": rate, "ops_per_sm_per_clk": rate / sms / (mhz.value * 1e6),
                          "sms": sms}), flush=True)


def run_batched_leg(dev, reps: int = 5):
    """The batched uneven workload: 64 instances (seeds 100-163, n from
    {20,50,100,200}, m from {5,10,20}, pools of 1,024 to 65,536 nodes).  One
    graph-replayed persistent launch over all pools against one autotuned
    plain launch per pool, same buffers, bit-exact."""
    import torch
    from paper_1208_3933_gb300 import fsp, workloads
    ws = workloads.batched_instances()
    insts = [fsp.Instance(w.p) for w in ws]
    bufs = [(torch.from_numpy(w.rows).to(dev), torch.from_numpy(w.depths).to(dev)) for w in ws]
    outs = [torch.empty(w.N, dtype=torch.int32, device=dev) for w in ws]
    outs_b = [torch.empty(w.N, dtype=torch.int32, device=dev) for w in ws]
    total = sum(w.N for w in ws)
    for inst, (r, d), o in zip(insts, bufs, outs):
        fsp.fsp_autotune(inst, r, d, o)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    def per_pool():
        for inst, (r, d), o in zip(insts, bufs, outs):
            fsp.fsp_bound_pool(inst, r, d, o)

    plain_ms = timed(per_pool)
    batch_pools = [(i, r, d, o) for i, (r, d), o in zip(insts, bufs, outs_b)]
    tuned_w, tuned_c, _ = fsp.fsp_batch_autotune_ex(batch_pools)
    with fsp.Batch(batch_pools, warps_per_block=tuned_w) as b:
        tile_only_ms = timed(b.launch_graph)
    with fsp.Batch(batch_pools, warps_per_block=tuned_w, couples_per_item=tuned_c) as b:
        batch_ms = timed(b.launch_graph)
        q = b.query()
    same = all(torch.equal(a, c) for a, c in zip(outs, outs_b))
    for inst in insts:
        inst.close()
    return {"workload": "64 instances, seeds 100-163", "pools": len(ws), "nodes": total,
            "batched_nodes_per_s": total / (batch_ms * 1e-3), "plain_nodes_per_s": total / (plain_ms * 1e-3),
            "batched_ms": batch_ms, "plain_ms": plain_ms, "speedup": plain_ms / batch_ms,
            "work_items": q["work_items"], "warps_per_block": q["warps_per_block"],
            "couples_per_item": q["couples_per_item"], "tile_only_ms": tile_only_ms,
            "tuned_shape": {"warps": tuned_w, "couples_per_item": tuned_c},
            "bit_exact_vs_plain": bool(same),
            "launch": "one CUDA-graph replay; warps per block and couples per work item autotuned"}


def run_pool_size_leg(fsp, inst, rows_d, dep_d, outs, stream, P: int, dep_h, n_jobs: int, m_mach: int,
                      peak: float, reps: int = 10):
    """Nodes/s against pool size on the same 200x20 instance (the paper varies
    the pool from 4,096 to 262,144 nodes): each size is a slice of the
    device-resident pool copies, a new slice every launch, timed with CUDA
    events; the default launch shape (batches split by couples while the pool
    leaves SMs idle) beside the same shape with every couple in one work item.
    Both shapes must give identical bounds.  Each size's roofline fraction
    is the algorithmic integer operations of its launches over their time,
    against the same ALU peak as the main line."""
    import torch
    total = rows_d[0].shape[0]
    out = []
    for N in (4096, 8192, 16384, 32768, 65536, 131072):
        shape = fsp.fsp_tuned_config(inst, N)
        whole = dict(shape, pairs_per_tile=P)
        # the shape fsp_autotune picks for this pool size (timed on the first slice)
        tuned, _ = fsp.fsp_autotune(inst, rows_d[0][:N], dep_d[0][:N], outs[0][:N], stream=stream)
        row = {"nodes": N, "launch": shape, "tuned_launch": tuned}
        for key, cfg in (("default", shape), ("one_work_item_per_batch", whole), ("tuned", tuned)):
            for i in range(3):
                fsp.fsp_bound_pool(inst, rows_d[i % 3][:N], dep_d[i % 3][:N], outs[i % 3][:N], stream=stream,
                                   config=cfg)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(reps):
                lo = (i * N) % (total - N + 1)
                c = i % 3
                fsp.fsp_bound_pool(inst, rows_d[c][lo:lo + N], dep_d[c][lo:lo + N], outs[c][lo:lo + N],
                                   stream=stream, config=cfg)
            e1.record(stream)
            torch.cuda.synchronize()
            secs = e0.elapsed_time(e1) * 1e-3
            row[key + "_nodes_per_s"] = N * reps / secs
            ops = sum(algorithmic_int_ops(n_jobs, m_mach, dep_h[(i * N) % (total - N + 1):][:N])
                      for i in range(reps))
            row[key + "_roofline_frac"] = ops / secs / peak
        a = fsp.fsp_bound_pool(inst, rows_d[0][:N], dep_d[0][:N], stream=stream, config=shape)
        b = fsp.fsp_bound_pool(inst, rows_d[0][:N], dep_d[0][:N], stream=stream, config=whole)
        c = fsp.fsp_bound_pool(inst, rows_d[0][:N], dep_d[0][:N], stream=stream, config=tuned)
        torch.cuda.synchronize()
        row["same_bounds"] = bool(torch.equal(a, b) and torch.equal(a, c))
        out.append(row)
    return out


def run_bnb_leg(seeds=(200, 201, 203, 202), node_limit: int = 50_000_000, expand: int = 256):
    """Whole searches of the serving workload (n=20, m=5), NEH upper bound:
    the host-driven DFS (branching on the host, one device pool per
    expansion), and the device-driven search (branching and elimination on
    the device, `expand` parents per round) in depth-first and best-first
    order.  Node counts, wall time and optimum checks against the optima the
    oracle stored in tests/golden."""
    from paper_1208_3933_gb300 import fsp, workloads
    gpath = os.path.join(ROOT, "tests", "golden", "serving_optima.json")
    golden = json.load(open(gpath))["results"] if os.path.exists(gpath) else {}
    probs = dict(workloads.serving_searches())
    out = []
    srv = fsp.Server()
    for seed in seeds:
        p = probs[seed]
        rec = golden.get(str(seed)) or {}
        with fsp.Instance(p) as inst:
            neh_ms = fsp.fsp_neh(inst)[0]
            row = {"seed": seed, "n": int(p.shape[0]), "m": int(p.shape[1]), "ub0_neh": int(neh_ms),
                   "optimum_stored": rec.get("opt")}
            runs = [("host_dfs", lambda: fsp.fsp_branch_and_bound(inst, neh_ms)),
                    ("device_dfs", lambda: fsp.fsp_branch_and_bound_device(inst, neh_ms, expand=expand,
                                                                           node_limit=node_limit)),
                    ("device_best_first", lambda: fsp.fsp_branch_and_bound_device(
                        inst, neh_ms, expand=expand, node_limit=node_limit, selection=fsp.FSP_SELECT_BEST_FIRST)),
                    ("server_8_searchers", lambda: srv.solve(inst, neh_ms, searchers=8, expand=64,
                                                             node_limit=node_limit)[:4])]
            for name, fn in runs:
                if name in ("host_dfs", "server_8_searchers") and seed == 202:
                    continue  # 12 M nodes through host-built pools: minutes
                t0 = time.perf_counter()
                st, best, _, nodes = fn()
                dt = time.perf_counter() - t0
                # status FSP_ENOTFOUND: NEH was optimal (nothing strictly better exists)
                found = best if st == fsp.FSP_OK else (neh_ms if st == fsp.FSP_ENOTFOUND else None)
                row[name] = {"status": int(st), "optimum": found, "nodes": int(nodes), "seconds": dt,
                             "nodes_per_s": nodes / dt if dt > 0 else None,
                             "matches_stored": (found == rec.get("opt")) if rec.get("opt") is not None else None}
        out.append(row)
    srv.close()
    return out


def run_config_leg(fsp, name: str, dev, peak: float, steps: int = 20, warmup: int = 3):
    """One more bounding configuration at full size -- 20x20 (65,536 nodes,
    seed 1) or 500x20 (65,536 nodes, seed 2, tiled staging) -- measured as
    the main line is: launch shape autotuned on the pool beforehand, every
    launch timed with CUDA events on its stream, the L2 flushed (a 256 MB
    write) between launches so no launch finds its pool in L2, and the
    roofline fraction = algorithmic integer operations / kernel time / ALU
    peak."""
    import torch
    from paper_1208_3933_gb300 import workloads
    w = workloads.named_pool(name)
    stream = torch.cuda.current_stream(dev)
    with fsp.Instance(w.p) as inst:
        r = torch.from_numpy(w.rows).to(dev)
        d = torch.from_numpy(w.depths).to(dev)
        out = torch.empty(w.N, dtype=torch.int32, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        _, tuned_ms = fsp.fsp_autotune(inst, r, d, out, stream=stream)
        launch = fsp.fsp_tuned_config(inst, w.N)
        for _ in range(warmup):
            fsp.fsp_bound_pool(inst, r, d, out, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 255)
            ev[i][0].record(stream)
            fsp.fsp_bound_pool(inst, r, d, out, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    ops = algorithmic_int_ops(w.n, w.m, w.depths)
    return {"workload": name, "n": w.n, "m": w.m, "nodes": w.N, "seed": w.seed, "nodes_per_s": w.N / (ms * 1e-3),
            "kernel_ms_mean": ms, "ops_per_launch": ops, "roofline_frac": ops / (ms * 1e-3) / peak,
            "launch": launch, "kernel": kernel_name(launch), "autotune_ms": tuned_ms,
            "l2": "256 MB write between launches"}


def run_sizes_leg(dev):
    """The pool-size and configuration legs alone (profiling): pool sizes
    4,096-131,072 of the 200x20 pool, then the 20x20 and 500x20 pools."""
    import torch
    from paper_1208_3933_gb300 import fsp
    w = rank_pool(0)
    props = torch.cuda.get_device_properties(dev)
    peak = alu_peak_ops(props.multi_processor_count, 2070.0, ALU_LANES_PER_SM)
    stream = torch.cuda.current_stream(dev)
    with fsp.Instance(w.p) as inst:
        rows_d = [torch.from_numpy(w.rows).to(dev) for _ in range(3)]
        dep_d = [torch.from_numpy(w.depths).to(dev) for _ in range(3)]
        outs = [torch.empty(w.N, dtype=torch.int32, device=dev) for _ in range(3)]
        sizes = run_pool_size_leg(fsp, inst, rows_d, dep_d, outs, stream, inst.info().pairs, w.depths, w.n, w.m,
                                  peak)
    configs = [run_config_leg(fsp, nm, dev, peak) for nm in ("pool_20x20", "pool_500x20")]
    return {"pool_sizes": sizes, "configs": configs}


def load_golden_optima():
    """Optima of the serving-loop searches stored by the oracle (tests/golden)."""
    gpath = os.path.join(ROOT, "tests", "golden", "serving_optima.json")
    if not os.path.exists(gpath):
        return {}
    return {int(k): v.get("opt") for k, v in json.load(open(gpath))["results"].items()}


def run_served_leg(node_limit: int = 500_000_000, expand: int = 1024, ig_iterations: int = 2000, slots: int = 8,
                   rate_hz: float = 100.0, pools_per_stream: int = 8):
    """The serving loop: 32 depth-first searches (n=20; m=5 for seeds 200-215,
    m=10 for 216-231) plus 16 streams of 200x20 pools (4,096-32,768 nodes,
    Poisson arrivals), run twice on identical work:
      served -- every search and stream submits its pools to one bounding
                server (continuous batching, admission by device footprint);
      plain  -- the same searches and streams, each pool bounded by its own
                plain launch (fsp_bound_pool_host on the client's stream).
    Each search starts from the library's iterated-greedy schedule (computed
    once, outside both arms) and is cut only by a stated node budget; the
    searches are deterministic, so both arms bound the same pools.  Reported:
    nodes/s of each arm (all nodes of both kinds over the arm's wall time),
    the server's p50/p99 pool latency, and every search's optimum against the
    optimum the oracle stored."""
    import threading

    import torch
    from paper_1208_3933_gb300 import fsp, workloads
    golden = load_golden_optima()
    searches = workloads.serving_searches()
    streams = workloads.serving_streams(rate_hz=rate_hz, pools_per_stream=pools_per_stream)
    s_insts = {s: fsp.Instance(p) for s, p in searches}
    st_insts = [fsp.Instance(p) for p, _ in streams]
    t0 = time.perf_counter()
    ub = {s: fsp.fsp_iterated_greedy(s_insts[s], iterations=ig_iterations, seed=s)[0] for s, _ in searches}
    ig_s = time.perf_counter() - t0

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    pools = [[(t, pinned(r), pinned(d), pinned(np.zeros(d.shape[0], np.int32))) for t, r, d in pl]
             for _, pl in streams]
    stream_nodes = sum(d.shape[0] for pl in pools for _, _, d, _ in pl)

    def arm(served: bool):
        results, lat = {}, []
        srv = fsp.Server(hbm_budget_bytes=4 << 30, slots=slots) if served else None
        errors = []

        def search(seed):
            try:
                if served:
                    results[seed] = srv.search(s_insts[seed], ub[seed], expand=expand, node_limit=node_limit)
                else:
                    results[seed] = fsp.fsp_search_plain(s_insts[seed], ub[seed], expand=expand,
                                                         node_limit=node_limit)
            except Exception as e:  # reported, never silently dropped
                errors.append(f"search {seed}: {e}")

        def stream(i):
            try:
                cs = None if served else torch.cuda.Stream()
                t_0 = time.perf_counter()
                reqs = []
                for t, r, d, o in pools[i]:
                    delay = t - (time.perf_counter() - t_0)
                    if delay > 0:
                        time.sleep(delay)
                    if served:
                        reqs.append(srv.submit(st_insts[i], r, d, out=o))
                    else:
                        a = time.perf_counter()
                        fsp.fsp_bound_pool_host(st_insts[i], r, d, o, stream=cs)
                        lat.append(time.perf_counter() - a)
                for q in reqs:
                    if q.wait(600_000_000) != fsp.FSP_OK:
                        errors.append(f"stream {i}: request failed")
                    q.release()
            except Exception as e:
                errors.append(f"stream {i}: {e}")

        threads = [threading.Thread(target=search, args=(s,)) for s, _ in searches]
        threads += [threading.Thread(target=stream, args=(i,)) for i in range(len(streams))]
        t_start = time.perf_counter()
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        wall = time.perf_counter() - t_start
        stats = srv.stats() if served else None
        if srv is not None:
            srv.close()
        outs = [o.copy() for pl in pools for _, _, _, o in pl]
        return results, wall, stats, lat, outs, errors

    s_res, s_wall, stats, _, s_outs, s_err = arm(True)
    p_res, p_wall, _, p_lat, p_outs, p_err = arm(False)
    per_seed, nodes_search = [], 0
    for seed, p in searches:
        st, best, _, nodes = s_res.get(seed, (None, None, None, 0))
        pst, pbest, _, pnodes = p_res.get(seed, (None, None, None, 0))
        nodes_search += nodes
        solved = st in (fsp.FSP_OK, fsp.FSP_ENOTFOUND)
        opt = (best if st == fsp.FSP_OK else ub[seed]) if solved else None
        per_seed.append({"seed": seed, "m": int(p.shape[1]), "ub0": ub[seed], "status": "solved" if solved else "cut",
                         "optimum": opt, "nodes": nodes, "oracle_optimum": golden.get(seed),
                         "plain_same": (st, best, nodes) == (pst, pbest, pnodes)})
    total = nodes_search + stream_nodes
    solved = [r for r in per_seed if r["status"] == "solved"]
    verified = [r["seed"] for r in solved if r["oracle_optimum"] is not None and r["optimum"] == r["oracle_optimum"]]
    wrong = [r["seed"] for r in solved if r["oracle_optimum"] is not None and r["optimum"] != r["oracle_optimum"]]
    unverified = [r["seed"] for r in solved if r["oracle_optimum"] is None]
    for inst in list(s_insts.values()) + st_insts:
        inst.close()
    return {"workload": "32 DFS searches (20x5 seeds 200-215, 20x10 seeds 216-231) + 16 Poisson streams of "
                        "200x20 pools", "node_budget_per_search": node_limit, "expand": expand, "slots": slots,
            "ub0": f"library iterated greedy, {ig_iterations} iterations per search ({ig_s:.1f} s, outside both arms)",
            "served_nodes_per_s": total / s_wall, "plain_nodes_per_s": total / p_wall,
            "served_over_plain": p_wall / s_wall, "nodes": total, "search_nodes": nodes_search,
            "stream_nodes": int(stream_nodes), "served_wall_s": s_wall, "plain_wall_s": p_wall,
            "p50_us": stats["p50_us"], "p99_us": stats["p99_us"], "pools": stats["pools_done"],
            "batches": stats["batches"], "mean_pools_per_batch": stats["mean_pools_per_batch"],
            "plain_stream_pool_p50_us": 1e6 * statistics.median(p_lat) if p_lat else None,
            "same_work": all(r["plain_same"] for r in per_seed) and all(np.array_equal(a, b)
                                                                        for a, b in zip(s_outs, p_outs)),
            "searches_solved": len(solved), "searches_cut": [r["seed"] for r in per_seed if r["status"] == "cut"],
            "optima_verified_vs_oracle": len(verified), "optima_unverified": unverified, "optima_wrong": wrong,
            "errors": s_err + p_err, "per_seed": per_seed}


def summarise(line: dict) -> dict:
    """Headline numbers of every leg, compact, for the end of the JSON line."""
    def r3(x):
        return None if x is None else float(f"{x:.3g}")

    out = {"pool_200x20": {"nodes_per_s": r3(line["value"]), "frac": r3(line["roofline"]["frac"])}}
    for c in line.get("configs") or []:
        out[c["workload"]] = {"nodes_per_s": r3(c["nodes_per_s"]), "frac": r3(c["roofline_frac"])}
    if line.get("pool_sizes"):
        out["pool_size_frac"] = {str(r["nodes"]): r3(max(r["default_roofline_frac"], r["tuned_roofline_frac"]))
                                 for r in line["pool_sizes"]}
    b = line.get("batched")
    if b:
        out["batched"] = {"nodes_per_s": r3(b["batched_nodes_per_s"]), "plain_nodes_per_s": r3(b["plain_nodes_per_s"]),
                          "speedup": r3(b["speedup"]), "bit_exact": b["bit_exact_vs_plain"],
                          "shape": b.get("tuned_shape")}
    v = line.get("served")
    if v:
        out["served"] = {"served_nodes_per_s": r3(v["served_nodes_per_s"]),
                         "plain_nodes_per_s": r3(v["plain_nodes_per_s"]),
                         "served_over_plain": r3(v["served_over_plain"]), "same_work": v["same_work"],
                         "p50_us": r3(v["p50_us"]), "p99_us": r3(v["p99_us"]),
                         "solved": f'{v["searches_solved"]}/32', "verified_vs_oracle": v["optima_verified_vs_oracle"],
                         "unverified": v["optima_unverified"], "wrong": v["optima_wrong"], "cut": v["searches_cut"],
                         "node_budget": v["node_budget_per_search"]}
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_pool(rank: int, name: str = WORKLOAD):
    from paper_1208_3933_gb300 import workloads
    w = workloads.named_pool(name)
    if rank == 0:
        return w
    rng = np.random.default_rng([2, rank])
    rows, depths = workloads.random_pool(rng, w.n, w.N)
    return workloads.PoolWorkload(w.name, w.n, w.m, w.seed, w.p, rows, depths)


def host_cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, else the Arm part),
    with the core count."""
    name = ""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part") and not name:
                name = line.split(":", 1)[1].strip()
    except OSError:
        pass
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    name = arm_parts.get(name.lower(), name)
    return f"{name or 'unknown'} x {os.cpu_count()}"


def cpu_oracle_rate(w, seconds: float = 2.0, threads: int | None = None, repeats: int = 3):
    """Times the oracle as it stands on a bounded sample of the pool, on all
    host cores (the single-threaded C routine on disjoint chunks): the best
    of `repeats` runs over the same sample, about `seconds` in all."""
    import oracle
    threads = threads or os.cpu_count() or 1
    t = oracle.Tables(w.p)
    probe = min(w.N, 64 * threads)
    t0 = time.perf_counter()
    t.lb_pool(w.rows[:probe], w.depths[:probe], threads=threads)
    rate = probe / max(time.perf_counter() - t0, 1e-9)
    sample = int(min(w.N, max(threads, rate * seconds / repeats)))
    best = float("inf")
    for _ in range(repeats):
        t0 = time.perf_counter()
        t.lb_pool(w.rows[:sample], w.depths[:sample], threads=threads)
        best = min(best, time.perf_counter() - t0)
    return sample / best, sample, best, threads


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, rank 0 only, on the same workload."""
    if rank != 0:
        return
    from paper_1208_3933_gb300 import workloads
    w = workloads.named_pool(WORKLOAD)
    threads = os.cpu_count() or 1
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rate(w, seconds=min(per_step, 2.0), threads=threads)
    rates, samples, secs = [], [], []
    for _ in range(args.steps):
        r, s, dt, _ = cpu_oracle_rate(w, seconds=min(per_step, 5.0), threads=threads)
        rates.append(r)
        samples.append(s)
        secs.append(dt)
    total_nodes, total_s = float(sum(samples)), float(sum(secs))
    value = total_nodes / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": w.n, "m": w.m, "nodes": w.N, "seed": w.seed},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {samples[0]} nodes of the 262,144-node pool per step, bounded by the "
                                   f"plain C oracle on {threads} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch
    from paper_1208_3933_gb300 import build, fsp

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = rank_pool(rank, args.workload)
    if args.nodes:
        from paper_1208_3933_gb300 import workloads
        w = workloads.PoolWorkload(w.name, w.n, w.m, w.seed, w.p, np.ascontiguousarray(w.rows[:args.nodes]),
                                   np.ascontiguousarray(w.depths[:args.nodes]))
    inst = fsp.Instance(w.p)
    copies = 3
    rows_d = [torch.from_numpy(w.rows).to(dev) for _ in range(copies)]
    dep_d = [torch.from_numpy(w.depths).to(dev) for _ in range(copies)]
    outs = [torch.empty(w.N, dtype=torch.int32, device=dev) for _ in range(copies)]
    stream = torch.cuda.current_stream(dev)

    # launch shape: forced (profiling) or autotuned on this pool, outside the timed region
    cfg = None
    if args.config:
        cfg = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.config.split(",") if kv}
        tuned_ms = None
    else:
        _, tuned_ms = fsp.fsp_autotune(inst, rows_d[0], dep_d[0], outs[0], stream=stream)
    launch = fsp.fsp_tuned_config(inst, w.N) if cfg is None else cfg

    for i in range(args.warmup):
        fsp.fsp_bound_pool(inst, rows_d[i % copies], dep_d[i % copies], outs[i % copies], stream=stream, config=cfg)
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    with sampler:
        time.sleep(0.3)
        barrier(world)
        torch.cuda.synchronize(dev)
        launches0 = fsp.fsp_kernel_launches()
        region0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            fsp.fsp_bound_pool(inst, rows_d[i % copies], dep_d[i % copies], outs[i % copies], stream=stream,
                               config=cfg)
            ev[i][1].record(stream)
        region1.record(stream)
        launches = fsp.fsp_kernel_launches() - launches0
        torch.cuda.synchronize(dev)
        barrier(world)
    region_ms = region0.elapsed_time(region1)
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    region_ms_max = max_over_ranks(world, region_ms)
    nodes_total = float(w.N) * args.steps * world
    value = nodes_total / (region_ms_max * 1e-3)

    # end to end through the C ABI with pinned host buffers: H2D of the pool,
    # bounding, D2H of the bounds, every step
    h_rows = torch.from_numpy(w.rows).pin_memory()
    h_dep = torch.from_numpy(w.depths).pin_memory()
    h_out = torch.empty(w.N, dtype=torch.int32).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        fsp.fsp_bound_pool_host(inst, h_rows, h_dep, h_out, stream=stream)
    barrier(world)
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fsp.fsp_bound_pool_host(inst, h_rows, h_dep, h_out, stream=stream)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = float(w.N) * e2e_steps * world / e2e_s
    ok_e2e = bool(np.array_equal(h_out.numpy(), outs[0].cpu().numpy()))

    if rank != 0:
        return
    clocks = sampler.summary()
    ops = algorithmic_int_ops(w.n, w.m, w.depths)
    mean_kernel_s = statistics.mean(kernel_ms) * 1e-3
    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks["sm_max_mhz"] or 2070.0
    peak = alu_peak_ops(props.multi_processor_count, sm_max, ALU_LANES_PER_SM)
    achieved = ops / mean_kernel_s
    # the CPU baseline is measured in the single-GPU run only
    cpu_rate, cpu_sample, cpu_s, cpu_threads = cpu_oracle_rate(w, seconds=2.0) if world == 1 else (0.0, 0, 0.0, 0)
    cpu1_rate, cpu1_sample, cpu1_s, _ = cpu_oracle_rate(w, seconds=1.0, threads=1) if world == 1 else (0.0, 0, 0.0, 0)
    info = inst.info()
    # the extra legs run once, in the single-GPU run
    extra = not (args.nodes or args.no_extra) and world == 1
    sizes = run_pool_size_leg(fsp, inst, rows_d, dep_d, outs, stream, info.pairs, w.depths, w.n, w.m,
                              peak) if extra else None
    configs = [run_config_leg(fsp, nm, dev, peak) for nm in ("pool_20x20", "pool_500x20")] if extra else None
    bnb = run_bnb_leg() if extra else None
    batched = run_batched_leg(dev) if extra else None
    served = run_served_leg() if extra else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": region_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "dtype_note": "integer bound; the couple scan runs one fused int32 add-max per entry on the slack "
                      "scaled by 1024 with the job in its low 10 bits, exact (every result equals the "
                      "oracle's int64)",
        "config": {"workload": w.name, "n": w.n, "m": w.m, "nodes_per_step_per_gpu": w.N, "seed": w.seed,
                   "p": "U[1,99]", "depth": "U{0..199}", "records": "compact" if info.compact else "wide",
                   "l2": "3 rotating pool copies of 105 MB (inputs larger than the 129 MB L2)",
                   "launch": launch, "autotune_ms": tuned_ms},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "int-ops/s",
                     "frac": achieved / peak, "traffic": read_traffic(w.N),
                     "peak_basis": f"{props.multi_processor_count} SMs x {ALU_LANES_PER_SM} int32 lanes x "
                                   f"{sm_max:.0f} MHz", "ops_per_launch": ops,
                     "kernel_ms_mean": mean_kernel_s * 1e3, "kernel": kernel_name(launch),
                     "timed": "CUDA events around each step's fsp_bound_pool on its stream: the bounding "
                              "kernel(s) of the launch shape plus, for pools of >= 8192 nodes and >= 64 jobs, the "
                              "two small depth-order kernels"},
        "cpu_baseline": None if world > 1 else {"value": cpu_rate, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": f"first {cpu_sample} nodes of the pool, plain C oracle on {cpu_threads} threads, "
                                   f"best of 3 runs of {cpu_s:.2f} s",
                         "single_thread": {"value": cpu1_rate, "sample": f"first {cpu1_sample} nodes, 1 thread, "
                                                                         f"best of 3 runs of {cpu1_s:.2f} s"},
                         "host_cpu": host_cpu_model()},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(w.rows.nbytes + w.depths.nbytes),
                "d2h_bytes_per_step": int(4 * w.N), "bit_exact_vs_device": ok_e2e},
        "gpu_launches": launches,
        "clocks": clocks,
        "pool_sizes": sizes,
        "bnb_searches": bnb,
        "configs": configs,
        "batched": batched,
        "served": served,
    }
    line["summary"] = summarise(line)  # last key: the end of the line holds every leg's headline
    print(json.dumps(line), flush=True)
    inst.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--nodes", type=int, default=0,
                    help="bound only the first NODES nodes of the pool (small profiling cases)")
    ap.add_argument("--alu-peak", action="store_true", help="run the integer-pipe throughput probe and exit")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--workload", default=WORKLOAD, choices=["pool_20x20", "pool_200x20", "pool_500x20"],
                    help="bound another pool as the main line (profiling; the benchmark is pool_200x20)")
    ap.add_argument("--leg", default="", choices=["", "batched", "served", "searches", "sizes"],
                    help="run one extra leg alone (single GPU) and print its JSON line (profiling)")
    ap.add_argument("--served-expand", type=int, default=0, help="served leg: parents per request (profiling)")
    ap.add_argument("--served-slots", type=int, default=0, help="served leg: server slots (profiling)")
    ap.add_argument("--served-budget", type=int, default=0, help="served leg: node budget per search (profiling)")
    ap.add_argument("--config", default="",
                    help="force a launch shape, e.g. kernel=2,warps_per_block=14 (profiling); default: autotuned")
    args = ap.parse_args()
    if args.alu_peak:
        run_alu_peak()
        return
    if args.leg:
        import torch
        from paper_1208_3933_gb300 import build
        build.build()
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        served_kw = {k: v for k, v in (("expand", args.served_expand), ("node_limit", args.served_budget),
                                       ("slots", args.served_slots)) if v}
        leg = {"batched": lambda: run_batched_leg(dev), "served": lambda: run_served_leg(**served_kw),
               "searches": run_bnb_leg, "sizes": lambda: run_sizes_leg(dev)}[args.leg]()
        print(json.dumps({"leg": args.leg, "result": leg}), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
