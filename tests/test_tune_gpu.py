"""The launch-shape autotuner: it picks a shape that fsp_bound_pool then
uses, all candidate shapes agree bit for bit (the tuner checks), and the
on-disk cache is read back without timing."""
import numpy as np
import pytest

import oracle
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,N", [(20, 5, 4000), (60, 20, 3000), (30, 10, 2500)])
def test_autotune_picks_a_shape_and_is_exact(gpu_lib, tmp_path, n, m, N):
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(n * 100 + m)
    p = rng.integers(1, 100, (n, m), dtype=np.int32)
    rows, depths = workloads.random_pool(rng, n, N, max_depth=n + 1)
    r = torch.from_numpy(rows).cuda()
    d = torch.from_numpy(depths).cuda()
    cache = str(tmp_path / "tune.txt")
    with fsp.Instance(p) as inst:
        before = fsp.fsp_tuned_config(inst, N)
        best, ms = fsp.fsp_autotune(inst, r, d, cache_path=cache)
        assert ms > 0 and best["kernel"] in (fsp.FSP_KERNEL_LOCKSTEP, fsp.FSP_KERNEL_LANES)
        assert fsp.fsp_tuned_config(inst, N) == best
        out = fsp.fsp_bound_pool(inst, r, d)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.Tables(p).lb_pool(rows, depths, threads=8))
        assert isinstance(before, dict)
    # a fresh instance of the same shape reads the cache and does no timing
    with fsp.Instance(p) as inst2:
        best2, ms2 = fsp.fsp_autotune(inst2, r, d, cache_path=cache)
        assert ms2 == -1.0 and best2 == best
