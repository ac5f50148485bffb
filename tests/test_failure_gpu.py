"""Failure paths on the GPU that fault nothing: a device-side wait that runs
out reports FSP_ETIMEDOUT through the instance's status word and the context
stays usable; bad rows and bad arguments come back as errors."""
import numpy as np
import pytest

import oracle
from paper_1208_3933_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_stays_usable(gpu_lib):
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(8)
    p = rng.integers(1, 100, (30, 8), dtype=np.int32)
    rows, depths = workloads.random_pool(rng, 30, 700, max_depth=31)
    with fsp.Instance(p) as inst:
        for limit in (1, 1000, 2_000_000):
            assert fsp.fsp_check_wait_timeout(inst, limit) == fsp.FSP_ETIMEDOUT
        out = fsp.fsp_bound_pool(inst, torch.from_numpy(rows).cuda(), torch.from_numpy(depths).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.Tables(p).lb_pool(rows, depths))
        assert fsp.fsp_check_wait_timeout(inst, 0) == fsp.FSP_EINVAL


def test_bad_launch_shapes_are_refused(gpu_lib):
    import torch
    fsp = gpu_lib
    rng = np.random.default_rng(9)
    p = rng.integers(1, 100, (40, 12), dtype=np.int32)
    rows, depths = workloads.random_pool(rng, 40, 100, max_depth=41)
    r, d = torch.from_numpy(rows).cuda(), torch.from_numpy(depths).cuda()
    with fsp.Instance(p) as inst:
        for cfg in (dict(kernel=3), dict(kernel=2, warps_per_block=17), dict(kernel=2, staging=6),
                    dict(kernel=2, staging=2, positions_per_tile=6), dict(kernel=2, blocks_per_sm=9),
                    dict(kernel=2, staging=5, warps_per_block=4, blocks_per_sm=5),
                    dict(kernel=2, staging=1, blocks_per_sm=3), dict(kernel=2, staging=3, blocks_per_sm=3)):
            with pytest.raises(fsp.FspError) as e:
                fsp.fsp_bound_pool(inst, r, d, config=cfg)
            assert e.value.status == fsp.FSP_EINVAL, cfg
        out = fsp.fsp_bound_pool(inst, r, d)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.Tables(p).lb_pool(rows, depths))
