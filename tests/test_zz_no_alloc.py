"""fsp_bound_batch_noalloc: the batched bound for callers that cannot allocate
memory when they need a bound (their GPU memory owned by another allocator,
or a loop that must not take cudaMalloc's synchronisation).  Its plan goes to
the kernel by value and its work counter lives in a fixed array inside the
library, so the test makes two calls in a row with different pools -- a
different count and order, an empty pool in the middle, sizes that are not a
multiple of 32, a per-job-release instance, invalid rows and instances of
different machine counts -- and checks every bound against the existing entry
point fsp_bound_pool and against the CPU oracle, bit for bit (the bounds are
integers).  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def _pool(w, N, bad_rows=0):
    rows, depths = w.rows[:N].copy(), w.depths[:N].copy()
    for i in range(bad_rows if N else 0):  # a repeated job, then a depth past n
        x = (7 * i + 3) % max(N, 1)
        if i % 2 == 0 and w.n > 1:
            depths[x] = max(depths[x], 2)
            rows[x, 1] = rows[x, 0]
        else:
            depths[x] = w.n + 1
    return rows, depths


def test_no_alloc_batch_matches_existing_entry_point_and_oracle_twice(gpu_lib):
    import torch
    fsp = gpu_lib
    lib = fsp.load()
    ws = workloads.batched_instances(range(100, 112))
    release = workloads.batched_instances([140])[0]
    insts = [fsp.Instance(w.p) for w in ws] + [fsp.Instance(release.p, flags=fsp.FSP_INSTANCE_RELEASE_PER_JOB)]
    ws = ws + [release]
    sizes_1 = [3000, 1000, 2048, 777, 31, 1500, 2600, 64, 33, 1200, 900, 2500, 1111]
    sizes_2 = [0, 2049, 5, 1800, 96, 0, 1024, 321, 2222, 17, 640, 1, 3001]
    calls = [
        [(i, sizes_1[i], 2 if i % 3 == 0 else 0) for i in range(len(ws))],
        [(i, sizes_2[i], 3 if i % 4 == 1 else 0) for i in reversed(range(len(ws)))][:11],
    ]
    for call, spec in enumerate(calls):
        pools, want_plain, want_oracle = [], [], []
        for i, N, bad in spec:
            w, inst = ws[i], insts[i]
            N = min(N, w.N)
            rows, depths = _pool(w, N, bad)
            r = torch.from_numpy(rows).cuda()
            d = torch.from_numpy(depths).cuda()
            o = torch.full((N,), -9, dtype=torch.int32, device="cuda")
            pools.append((inst, r, d, o))
            plain = fsp.fsp_bound_pool(inst, r, d)
            want_plain.append(plain)
            k = min(N, 200)  # the oracle checks the first nodes of every pool
            rel = oracle.RELEASE_EST if w is release else oracle.RELEASE_HEADS
            want_oracle.append(oracle.Tables(w.p).lb_pool(rows[:k], depths[:k], threads=8, release=rel))
        torch.cuda.synchronize()
        descs = (fsp.fsp_pool_desc * len(pools))()
        for i, (inst, r, d, o) in enumerate(pools):
            descs[i] = fsp.fsp_pool_desc(inst.handle.value, r.data_ptr() if r.numel() else None,
                                         d.data_ptr() if d.numel() else None,
                                         o.data_ptr() if o.numel() else None, r.shape[0])
        st = lib.fsp_bound_batch_noalloc(descs, len(pools),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == fsp.FSP_OK, fsp.fsp_status_string(st)
        torch.cuda.synchronize()
        for (i, N, bad), (inst, r, d, o), plain, orc in zip(spec, pools, want_plain, want_oracle):
            got = o.cpu().numpy()
            assert np.array_equal(got, plain.cpu().numpy()), (call, ws[i].name)
            assert np.array_equal(got[:orc.shape[0]], orc), (call, ws[i].name)
            if bad and got.size:
                assert (got == fsp.FSP_LB_INVALID).any(), (call, ws[i].name)
    # beyond the stated maximum the call is refused before any work
    too_many = (fsp.fsp_pool_desc * (fsp.FSP_NOALLOC_MAX_POOLS + 1))()
    assert lib.fsp_bound_batch_noalloc(too_many, fsp.FSP_NOALLOC_MAX_POOLS + 1, None) == fsp.FSP_EINVAL
    for inst in insts:
        inst.close()
