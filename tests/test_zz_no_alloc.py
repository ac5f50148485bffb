"""fsp_bound_batch_noalloc: the batched bound for callers that cannot allocate
memory (their GPU memory owned by another allocator, or a loop that must not
take cudaMalloc's synchronisation).  Its plan and work counter live in a fixed
array inside the library, so the test checks two calls in a row against the
existing entry points: every bound equal, bit for bit (the bounds are
integers).  This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_no_alloc_batch_matches_existing_entry_points_twice(gpu_lib):
    import torch
    fsp = gpu_lib
    ws = workloads.batched_instances(range(100, 110))
    insts = [fsp.Instance(w.p) for w in ws]
    bufs = [(torch.from_numpy(w.rows[:3000].copy()).cuda(), torch.from_numpy(w.depths[:3000].copy()).cuda())
            for w in ws]
    ref = []
    for inst, (r, d) in zip(insts, bufs):
        ref.append(fsp.fsp_bound_pool(inst, r, d))
    torch.cuda.synchronize()
    ref = [o.cpu().numpy() for o in ref]
    outs = [torch.full((r.shape[0],), -9, dtype=torch.int32, device="cuda") for r, _ in bufs]
    pools = [(inst, r, d, o) for inst, (r, d), o in zip(insts, bufs, outs)]
    lib = fsp.load()
    for call in range(2):
        for o in outs:
            o.fill_(-9)
        descs = (fsp.fsp_pool_desc * len(pools))()
        for i, (inst, r, d, o) in enumerate(pools):
            descs[i] = fsp.fsp_pool_desc(inst.handle.value, r.data_ptr(), d.data_ptr(), o.data_ptr(), r.shape[0])
        st = lib.fsp_bound_batch_noalloc(descs, len(pools),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == fsp.FSP_OK, fsp.fsp_status_string(st)
        torch.cuda.synchronize()
        for w, o, want in zip(ws, outs, ref):
            assert np.array_equal(o.cpu().numpy(), want), (call, w.name)
    # beyond the stated maximum the call is refused before any work
    too_many = (fsp.fsp_pool_desc * (fsp.FSP_NOALLOC_MAX_POOLS + 1))()
    assert lib.fsp_bound_batch_noalloc(too_many, fsp.FSP_NOALLOC_MAX_POOLS + 1, None) == fsp.FSP_EINVAL
    for inst in insts:
        inst.close()
