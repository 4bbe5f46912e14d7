"""Query sharding (paper_1511_02186_gb300.sharding) with the library as each rank's compute, on
the one GPU this process has: the ranks' contiguous query ranges are interpolated one after the
other (without gathering, so no process group is needed), and together they cover every query
once and match the FP64 oracle within the FP32 tolerance."""
import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, sharding, workloads
from parity import TOL_F32, oracle_for, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_cover_the_queries_and_match_the_oracle(world):
    import torch
    wl = workloads.small_case(51, 30000, 20001, k=10, pattern="clustered")
    with aidw.Context(0) as ctx:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
        p = aidw.default_params(k=wl.k)
        z = np.full(wl.m, np.nan)
        covered = np.zeros(wl.m, dtype=np.int32)
        for rank in range(world):
            b, e, part = sharding.interpolate_on_rank(ctx, ds, qx, qy, p, rank, world)
            torch.cuda.synchronize()
            z[b:e] = part["z"].cpu().numpy()
            covered[b:e] += 1
        ds.destroy()
    assert np.all(covered == 1)
    ref, _ = oracle_for(wl, aidw.F32C)
    assert rel_err(z, ref).max() <= TOL_F32
