"""Thin Python binding of the C ABI in include/fsp.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
buffers are torch CUDA tensors (PyTorch supplies memory and streams); all
bounding work runs in libfsp_gb300.so.  There is no CPU fallback: if the
library is missing or a CUDA device is absent the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsp_gb300.so")

FSP_OK = 0
FSP_EINVAL = -1
FSP_ENOMEM = -2
FSP_ECUDA = -3
FSP_EBADNODE = -4
FSP_ETIMEDOUT = -5
FSP_ENOTFOUND = -6
FSP_EBUSY = -7
FSP_LB_INVALID = -1
FSP_MAX_JOBS = 1024
FSP_MAX_MACHINES = 32

_lock = threading.Lock()
_lib = None


class FspError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {fsp_status_string(status)} ({status})")


class fsp_instance_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("pairs", ctypes.c_int32),
                ("compact", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("device", ctypes.c_int32), ("flags", ctypes.c_int32)]


FSP_INSTANCE_RELEASE_PER_JOB = 0x1  # release times read per job (fsp_instance_create_ex)

FSP_KERNEL_AUTO = 0
FSP_KERNEL_LOCKSTEP = 1
FSP_KERNEL_LANES = 2
FSP_STAGING_AUTO = 0
FSP_STAGING_RESIDENT = 1
FSP_STAGING_STREAMED = 2
FSP_STAGING_SPLIT = 3
FSP_STAGING_WARP = 4
FSP_STAGING_GLOBAL = 5


class fsp_launch_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("nodes_per_thread", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("pairs_per_tile", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("positions_per_tile", ctypes.c_int32),
                ("staging", ctypes.c_int32), ("tail_slices", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class fsp_pool_desc(ctypes.Structure):
    _fields_ = [("inst", ctypes.c_void_p), ("nodes", ctypes.c_void_p), ("depths", ctypes.c_void_p),
                ("out_lb", ctypes.c_void_p), ("N", ctypes.c_int64)]


class fsp_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_batch_pools", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("warps_per_block", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fsp_server_stats(ctypes.Structure):
    _fields_ = [("pools_done", ctypes.c_int64), ("nodes_done", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_pools_per_batch", ctypes.c_double), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("active_seconds", ctypes.c_double), ("queued", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("arena_bytes", ctypes.c_int64), ("arena_bytes_used", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def launch_config(**fields) -> fsp_launch_config:
    """fsp_launch_config from keyword fields (missing ones are 0 = choose)."""
    cfg = fsp_launch_config()
    for k, v in fields.items():
        setattr(cfg, k, int(v))
    return cfg


def load():
    """Opens libfsp_gb300.so (built in-tree by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        i32p = ctypes.POINTER(ctypes.c_int32)
        i16p = ctypes.POINTER(ctypes.c_int16)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sig = {
            "fsp_instance_create": ([i32p, i32, i32, ctypes.POINTER(vp)], i32),
            "fsp_instance_create_ex": ([i32p, i32, i32, ctypes.c_uint32, ctypes.POINTER(vp)], i32),
            "fsp_instance_destroy": ([vp], None),
            "fsp_instance_query": ([vp, ctypes.POINTER(fsp_instance_info)], i32),
            "fsp_bound_pool": ([vp, vp, vp, i64, vp, vp], i32),
            "fsp_bound_pool_ex": ([vp, vp, vp, i64, vp, vp, ctypes.POINTER(fsp_launch_config)], i32),
            "fsp_bound_pool_host": ([vp, vp, vp, i64, vp, vp], i32),
            "fsp_branch_and_bound": ([vp, i32, i16p, i32p, i64p], i32),
            "fsp_branch_and_bound_device": ([vp, i32, i32, i32, i64, i16p, i32p, i64p], i32),
            "fsp_autotune": ([vp, vp, vp, i64, vp, vp, ctypes.c_char_p, ctypes.POINTER(fsp_launch_config),
                              ctypes.POINTER(ctypes.c_float)], i32),
            "fsp_tuned_config": ([vp, i64, ctypes.POINTER(fsp_launch_config)], i32),
            "fsp_batch_create": ([ctypes.POINTER(fsp_pool_desc), i32, i32, ctypes.POINTER(vp)], i32),
            "fsp_batch_create_ex": ([ctypes.POINTER(fsp_pool_desc), i32, i32, i32, ctypes.POINTER(vp)], i32),
            "fsp_batch_query_ex": ([vp, i64p, i64p, i32p, i32p, i32p], i32),
            "fsp_batch_autotune_ex": ([ctypes.POINTER(fsp_pool_desc), i32, vp, i32p, i32p,
                                       ctypes.POINTER(ctypes.c_float)], i32),
            "fsp_batch_launch": ([vp, vp], i32),
            "fsp_batch_launch_graph": ([vp, vp], i32),
            "fsp_batch_query": ([vp, i64p, i64p, i32p, i32p], i32),
            "fsp_batch_destroy": ([vp], None),
            "fsp_batch_autotune": ([ctypes.POINTER(fsp_pool_desc), i32, vp, i32p, ctypes.POINTER(ctypes.c_float)],
                                   i32),
            "fsp_bound_batch_noalloc": ([ctypes.POINTER(fsp_pool_desc), i32, vp], i32),
            "fsp_server_create": ([ctypes.POINTER(fsp_server_config), ctypes.POINTER(vp)], i32),
            "fsp_server_submit": ([vp, vp, vp, vp, i64, vp, ctypes.POINTER(vp)], i32),
            "fsp_request_wait": ([vp, i64], i32),
            "fsp_request_cancel": ([vp], i32),
            "fsp_request_release": ([vp], None),
            "fsp_server_get_stats": ([vp, ctypes.POINTER(fsp_server_stats)], i32),
            "fsp_server_reset_stats": ([vp], i32),
            "fsp_server_shutdown": ([vp], i32),
            "fsp_server_destroy": ([vp], None),
            "fsp_server_search": ([vp, vp, i32, i32, i64, i16p, i32p, i64p], i32),
            "fsp_server_solve": ([vp, vp, i32, i32, i32, i64, i16p, i32p, i64p, i64p], i32),
            "fsp_neh": ([vp, i16p, i32p], i32),
            "fsp_iterated_greedy": ([vp, i32, ctypes.c_uint64, i16p, i32p], i32),
            "fsp_status_string": ([i32], ctypes.c_char_p),
            "fsp_version": ([], ctypes.c_char_p),
            "fsp_kernel_launches": ([], i64),
            "fsp_check_wait_timeout": ([vp, i64], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def fsp_status_string(status: int) -> str:
    return load().fsp_status_string(int(status)).decode()


def fsp_version() -> str:
    return load().fsp_version().decode()


def fsp_check_wait_timeout(inst: Instance, limit_cycles: int = 2_000_000) -> int:
    """Runs one device-side bounded wait that nothing completes; returns the
    status (FSP_ETIMEDOUT when the timeout path works)."""
    return int(load().fsp_check_wait_timeout(inst.handle, int(limit_cycles)))


def fsp_kernel_launches() -> int:
    """Kernels the library has enqueued in this process so far."""
    return int(load().fsp_kernel_launches())


def _check(status: int, where: str):
    if status != FSP_OK:
        raise FspError(status, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Instance:
    """Owns one fsp_instance (the processing times and every table of the
    bound, resident on the current CUDA device)."""

    def __init__(self, p, flags: int = 0):
        lib = load()
        p = np.ascontiguousarray(np.asarray(p), dtype=np.int32)
        if p.ndim != 2:
            raise ValueError("p must be a [n][m] matrix")
        self.p = p
        self.n, self.m = int(p.shape[0]), int(p.shape[1])
        self.flags = int(flags)
        h = ctypes.c_void_p()
        _check(lib.fsp_instance_create_ex(p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.n, self.m,
                                          self.flags, ctypes.byref(h)), "fsp_instance_create_ex")
        self._h = h

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("instance is destroyed")
        return self._h

    def info(self) -> fsp_instance_info:
        out = fsp_instance_info()
        _check(load().fsp_instance_query(self.handle, ctypes.byref(out)), "fsp_instance_query")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fsp_instance_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fsp_instance_create(p) -> Instance:
    return Instance(p)


def fsp_instance_destroy(inst: Instance) -> None:
    inst.close()


def _check_pool(inst: Instance, nodes, depths, out):
    import torch
    N = int(depths.shape[0])
    for name, t, dt in (("nodes", nodes, torch.int16), ("depths", depths, torch.int32), ("out_lb", out, torch.int32)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if tuple(nodes.shape) != (N, inst.n) or tuple(out.shape) != (N,):
        raise ValueError("nodes must be [N][n], depths and out_lb [N]")
    return N


def fsp_bound_pool(inst: Instance, nodes, depths, out=None, stream=None, config=None):
    """Bounds a device-resident pool; returns out (a new int32 tensor if None).
    Stream-ordered on ``stream`` (default: torch's current stream)."""
    import torch
    if out is None:
        out = torch.empty(depths.shape[0], dtype=torch.int32, device=depths.device)
    N = _check_pool(inst, nodes, depths, out)
    lib = load()
    if config is None:
        st = lib.fsp_bound_pool(inst.handle, ctypes.c_void_p(nodes.data_ptr()), ctypes.c_void_p(depths.data_ptr()),
                                N, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
        _check(st, "fsp_bound_pool")
    else:
        cfg = config if isinstance(config, fsp_launch_config) else launch_config(**dict(config))
        st = lib.fsp_bound_pool_ex(inst.handle, ctypes.c_void_p(nodes.data_ptr()),
                                   ctypes.c_void_p(depths.data_ptr()), N, ctypes.c_void_p(out.data_ptr()),
                                   _stream_handle(stream), ctypes.byref(cfg))
        _check(st, "fsp_bound_pool_ex")
    return out


def fsp_autotune(inst: Instance, nodes, depths, out=None, stream=None, cache_path=None):
    """Times every launch shape on this pool, keeps the fastest for N in the
    instance; returns (config dict, ms per launch or -1 if cached)."""
    import torch
    if out is None:
        out = torch.empty(depths.shape[0], dtype=torch.int32, device=depths.device)
    N = _check_pool(inst, nodes, depths, out)
    best = fsp_launch_config()
    ms = ctypes.c_float(0)
    st = load().fsp_autotune(inst.handle, ctypes.c_void_p(nodes.data_ptr()), ctypes.c_void_p(depths.data_ptr()), N,
                             ctypes.c_void_p(out.data_ptr()), _stream_handle(stream),
                             cache_path.encode() if cache_path else None, ctypes.byref(best), ctypes.byref(ms))
    _check(st, "fsp_autotune")
    return best.as_dict(), float(ms.value)


def fsp_tuned_config(inst: Instance, N: int) -> dict:
    cfg = fsp_launch_config()
    _check(load().fsp_tuned_config(inst.handle, int(N), ctypes.byref(cfg)), "fsp_tuned_config")
    return cfg.as_dict()


def fsp_bound_pool_host(inst: Instance, nodes, depths, out=None, stream=None):
    """Bounds a host-resident pool (numpy arrays or CPU tensors, pinned or
    pageable): copies in, bounds, copies back; returns when out is filled."""
    def host_ptr(a, dt):
        if hasattr(a, "data_ptr"):  # torch CPU tensor
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors")
            return ctypes.c_void_p(a.data_ptr()), a
        a = np.ascontiguousarray(a, dtype=dt)
        return ctypes.c_void_p(a.ctypes.data), a

    n_ptr, nodes = host_ptr(nodes, np.int16)
    d_ptr, depths = host_ptr(depths, np.int32)
    N = int(depths.shape[0])
    if tuple(nodes.shape) != (N, inst.n):
        raise ValueError("nodes must be [N][n]")
    if out is None:
        out = np.empty(N, np.int32)
    o_ptr, out = host_ptr(out, np.int32)
    if tuple(out.shape) != (N,):
        raise ValueError("out_lb must be [N]")
    st = load().fsp_bound_pool_host(inst.handle, n_ptr, d_ptr, N, o_ptr, _stream_handle(stream))
    _check(st, "fsp_bound_pool_host")
    return out


def fsp_branch_and_bound(inst: Instance, ub0: int):
    """Returns (status, best_makespan, best_perm, nodes_bounded); status is
    FSP_OK or FSP_ENOTFOUND (other failures raise)."""
    perm = np.zeros(inst.n, np.int16)
    best = ctypes.c_int32(0)
    nodes = ctypes.c_int64(0)
    st = load().fsp_branch_and_bound(inst.handle, int(ub0), perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)),
                                     ctypes.byref(best), ctypes.byref(nodes))
    if st not in (FSP_OK, FSP_ENOTFOUND):
        raise FspError(st, "fsp_branch_and_bound")
    return st, int(best.value), perm, int(nodes.value)


FSP_SELECT_DEPTH_FIRST = 0
FSP_SELECT_BEST_FIRST = 1


def fsp_branch_and_bound_device(inst: Instance, ub0: int, expand: int = 0, node_limit: int = 0,
                                selection: int = FSP_SELECT_DEPTH_FIRST):
    """B&B with branching and elimination on the device.  Returns (status,
    best_makespan, best_perm, nodes_bounded); status is FSP_OK,
    FSP_ENOTFOUND or FSP_ETIMEDOUT (other failures raise)."""
    perm = np.zeros(inst.n, np.int16)
    best = ctypes.c_int32(0)
    nodes = ctypes.c_int64(0)
    st = load().fsp_branch_and_bound_device(inst.handle, int(ub0), int(expand), int(selection), int(node_limit),
                                            perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)),
                                            ctypes.byref(best), ctypes.byref(nodes))
    if st not in (FSP_OK, FSP_ENOTFOUND, FSP_ETIMEDOUT):
        raise FspError(st, "fsp_branch_and_bound_device")
    return st, int(best.value), perm, int(nodes.value)


class Batch:
    """Owns one fsp_batch plan over pools given as (instance, nodes, depths,
    out) with torch CUDA tensors; keeps them alive while the plan exists."""

    def __init__(self, pools, warps_per_block: int = 0, couples_per_item: int = 0):
        lib = load()
        self._keep = list(pools)
        descs = (fsp_pool_desc * max(1, len(pools)))()
        for i, (inst, nodes, depths, out) in enumerate(pools):
            N = _check_pool(inst, nodes, depths, out)
            descs[i] = fsp_pool_desc(inst.handle.value, nodes.data_ptr(), depths.data_ptr(), out.data_ptr(), N)
        h = ctypes.c_void_p()
        _check(lib.fsp_batch_create_ex(descs, len(pools), int(warps_per_block), int(couples_per_item),
                                       ctypes.byref(h)), "fsp_batch_create_ex")
        self._h = h

    def launch(self, stream=None):
        _check(load().fsp_batch_launch(self._h, _stream_handle(stream)), "fsp_batch_launch")

    def launch_graph(self, stream=None):
        _check(load().fsp_batch_launch_graph(self._h, _stream_handle(stream)), "fsp_batch_launch_graph")

    def query(self) -> dict:
        items, nodes = ctypes.c_int64(), ctypes.c_int64()
        warps, blocks, cpi = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().fsp_batch_query_ex(self._h, ctypes.byref(items), ctypes.byref(nodes), ctypes.byref(warps),
                                         ctypes.byref(blocks), ctypes.byref(cpi)), "fsp_batch_query_ex")
        return dict(work_items=items.value, nodes=nodes.value, warps_per_block=warps.value, blocks=blocks.value,
                    couples_per_item=cpi.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fsp_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fsp_batch_create(pools, warps_per_block: int = 0, couples_per_item: int = 0) -> Batch:
    return Batch(pools, warps_per_block, couples_per_item)


def fsp_batch_autotune(pools, stream=None):
    """Fastest warps_per_block for a batch of (instance, nodes, depths, out)
    pools (torch CUDA tensors); returns (warps_per_block, ms per launch)."""
    lib = load()
    descs = (fsp_pool_desc * max(1, len(pools)))()
    for i, (inst, nodes, depths, out) in enumerate(pools):
        N = _check_pool(inst, nodes, depths, out)
        descs[i] = fsp_pool_desc(inst.handle.value, nodes.data_ptr(), depths.data_ptr(), out.data_ptr(), N)
    w, ms = ctypes.c_int32(), ctypes.c_float()
    _check(lib.fsp_batch_autotune(descs, len(pools), _stream_handle(stream), ctypes.byref(w), ctypes.byref(ms)),
           "fsp_batch_autotune")
    return int(w.value), float(ms.value)


def fsp_batch_autotune_ex(pools, stream=None):
    """Fastest (warps_per_block, couples_per_item) for a batch of (instance,
    nodes, depths, out) pools; returns (warps, couples per item, ms)."""
    lib = load()
    descs = (fsp_pool_desc * max(1, len(pools)))()
    for i, (inst, nodes, depths, out) in enumerate(pools):
        N = _check_pool(inst, nodes, depths, out)
        descs[i] = fsp_pool_desc(inst.handle.value, nodes.data_ptr(), depths.data_ptr(), out.data_ptr(), N)
    w, c, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(lib.fsp_batch_autotune_ex(descs, len(pools), _stream_handle(stream), ctypes.byref(w), ctypes.byref(c),
                                     ctypes.byref(ms)), "fsp_batch_autotune_ex")
    return int(w.value), int(c.value), float(ms.value)


FSP_NOALLOC_MAX_POOLS = 64


def fsp_bound_batch_noalloc(pools, stream=None):
    """Batched bound with no allocation inside the library (see include/fsp.h):
    pools are (instance, nodes, depths, out) with torch CUDA tensors."""
    descs = (fsp_pool_desc * max(1, len(pools)))()
    for i, (inst, nodes, depths, out) in enumerate(pools):
        N = _check_pool(inst, nodes, depths, out)
        descs[i] = fsp_pool_desc(inst.handle.value, nodes.data_ptr(), depths.data_ptr(), out.data_ptr(), N)
    _check(load().fsp_bound_batch_noalloc(descs, len(pools), _stream_handle(stream)), "fsp_bound_batch_noalloc")


class Request:
    """A pending fsp_server request; keeps its host buffers alive.  The
    handle dies with its server (fsp_server_destroy frees it)."""

    def __init__(self, handle, keep, server):
        self._h = handle
        self._keep = keep
        self._server = server

    @property
    def out(self):
        return self._keep[2]

    def _handle(self):
        if self._h is None or self._server._h is None:
            raise RuntimeError("request handle is released or its server is destroyed")
        return self._h

    def wait(self, timeout_us: int = -1) -> int:
        """fsp_request_wait: returns the status (FSP_OK, FSP_ETIMEDOUT, ...)."""
        return load().fsp_request_wait(self._handle(), int(timeout_us))

    def cancel(self) -> int:
        return load().fsp_request_cancel(self._handle())

    def release(self):
        if self._h is not None and self._h.value and self._server._h is not None:
            load().fsp_request_release(self._h)
        self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Server:
    """Owns an fsp_server (continuous-batching bounding server)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_batch_pools: int = 0, slots: int = 0,
                 warps_per_block: int = 0):
        cfg = fsp_server_config(int(hbm_budget_bytes), int(max_batch_pools), int(slots), int(warps_per_block), 0)
        h = ctypes.c_void_p()
        _check(load().fsp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "fsp_server_create")
        self._h = h

    def submit(self, inst: Instance, nodes, depths, out=None) -> Request:
        """Queues a host pool (numpy arrays, ideally in pinned memory)."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int16)
        depths = np.ascontiguousarray(depths, dtype=np.int32)
        N = int(depths.shape[0])
        if nodes.shape != (N, inst.n):
            raise ValueError("nodes must be [N][n]")
        if out is None:
            out = np.empty(N, np.int32)
        req = ctypes.c_void_p()
        st = load().fsp_server_submit(self._h, inst.handle, ctypes.c_void_p(nodes.ctypes.data),
                                      ctypes.c_void_p(depths.ctypes.data), N, ctypes.c_void_p(out.ctypes.data),
                                      ctypes.byref(req))
        _check(st, "fsp_server_submit")
        return Request(req, (nodes, depths, out), self)

    def stats(self) -> dict:
        st = fsp_server_stats()
        _check(load().fsp_server_get_stats(self._h, ctypes.byref(st)), "fsp_server_get_stats")
        return st.as_dict()

    def reset_stats(self):
        _check(load().fsp_server_reset_stats(self._h), "fsp_server_reset_stats")

    def shutdown(self):
        _check(load().fsp_server_shutdown(self._h), "fsp_server_shutdown")

    def search(self, inst: Instance, ub0: int, expand: int = 64, node_limit: int = 0):
        """fsp_server_search: (status, best_makespan, best_perm, nodes_bounded);
        status FSP_OK, FSP_ENOTFOUND, or FSP_ETIMEDOUT when node_limit cut it."""
        perm = np.zeros(inst.n, np.int16)
        best = ctypes.c_int32(0)
        nodes = ctypes.c_int64(0)
        st = load().fsp_server_search(self._h, inst.handle, int(ub0), int(expand), int(node_limit),
                                      perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), ctypes.byref(best),
                                      ctypes.byref(nodes))
        if st not in (FSP_OK, FSP_ENOTFOUND, FSP_ETIMEDOUT):
            raise FspError(st, "fsp_server_search")
        return st, int(best.value), perm, int(nodes.value)

    def solve(self, inst: Instance, ub0: int, searchers: int = 8, expand: int = 64, node_limit: int = 0):
        """fsp_server_solve: (status, best_makespan, best_perm, nodes_bounded,
        steals) of `searchers` cooperating searches sharing one incumbent."""
        perm = np.zeros(inst.n, np.int16)
        best = ctypes.c_int32(0)
        nodes = ctypes.c_int64(0)
        steals = ctypes.c_int64(0)
        st = load().fsp_server_solve(self._h, inst.handle, int(ub0), int(searchers), int(expand), int(node_limit),
                                     perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), ctypes.byref(best),
                                     ctypes.byref(nodes), ctypes.byref(steals))
        if st not in (FSP_OK, FSP_ENOTFOUND, FSP_ETIMEDOUT):
            raise FspError(st, "fsp_server_solve")
        return st, int(best.value), perm, int(nodes.value), int(steals.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fsp_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fsp_neh(inst: Instance):
    """NEH heuristic schedule: (makespan, perm)."""
    perm = np.zeros(inst.n, np.int16)
    mk = ctypes.c_int32(0)
    _check(load().fsp_neh(inst.handle, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), ctypes.byref(mk)),
           "fsp_neh")
    return int(mk.value), perm


def fsp_search_plain(inst: Instance, ub0: int, expand: int = 64, node_limit: int = 0):
    """fsp_server_search with no server: the same depth-first search, each
    pool bounded by its own plain launch (fsp_bound_pool_host).  Returns
    (status, best_makespan, best_perm, nodes_bounded)."""
    perm = np.zeros(inst.n, np.int16)
    best = ctypes.c_int32(0)
    nodes = ctypes.c_int64(0)
    st = load().fsp_server_search(None, inst.handle, int(ub0), int(expand), int(node_limit),
                                  perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), ctypes.byref(best),
                                  ctypes.byref(nodes))
    if st not in (FSP_OK, FSP_ENOTFOUND, FSP_ETIMEDOUT):
        raise FspError(st, "fsp_server_search")
    return st, int(best.value), perm, int(nodes.value)


def fsp_iterated_greedy(inst: Instance, iterations: int = 2000, seed: int = 0):
    """Iterated greedy heuristic schedule: (makespan, perm)."""
    perm = np.zeros(inst.n, np.int16)
    mk = ctypes.c_int32(0)
    _check(load().fsp_iterated_greedy(inst.handle, int(iterations), int(seed),
                                      perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), ctypes.byref(mk)),
           "fsp_iterated_greedy")
    return int(mk.value), perm
