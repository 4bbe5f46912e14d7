"""Failure path of the bounded on-device waits, without any GPU fault: a kernel waits with the
scans' own wait code on something that never completes, gives up after a short poll limit,
raises the context's error word and returns. The host must read AIDW_ERR_TIMEOUT, the error
must clear once read, and the context must keep working."""
import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32, oracle_for, params_of, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1], ids=["mbarrier", "counter"])
def test_expired_wait_reports_timeout_and_context_survives(which):
    with aidw.Context(0) as ctx:
        assert ctx.check_device_errors() == aidw.OK
        ctx.expire_wait(which, 4096)
        assert ctx.check_device_errors() == aidw.ERR_TIMEOUT
        assert ctx.check_device_errors() == aidw.OK  # read once, then clear
        # A synchronous call (host arrays) after an expired wait reports it ...
        wl = workloads.small_case(81, 3000, 700, k=10, pattern="clustered", side=50.0)
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        src = wl.as_f32()
        ctx.expire_wait(which, 4096)
        with pytest.raises(aidw.AidwError) as e:
            ctx.interpolate(ds, src.qx, src.qy, params_of(wl, aidw.F32C))
        assert e.value.status == aidw.ERR_TIMEOUT
        # ... and the next one runs normally.
        out, _, _ = ctx.interpolate(ds, src.qx, src.qy, params_of(wl, aidw.F32C))
        ref, _ = oracle_for(wl, aidw.F32C)
        assert rel_err(np.asarray(out, dtype=np.float64), ref).max() <= TOL_F32
        ds.destroy()


def test_expire_wait_rejects_bad_arguments():
    with aidw.Context(0) as ctx:
        for which, polls in ((2, 10), (-1, 10), (0, 0), (1, (1 << 20) + 1)):
            with pytest.raises(aidw.AidwError):
                ctx.expire_wait(which, polls)
        assert ctx.check_device_errors() == aidw.OK


def test_pipe_rate_probes_are_plausible():
    """The microbenchmarks behind the roofline denominators: every rate positive and below the
    SM's lane count, SM clock in a GB300 range."""
    with aidw.Context(0) as ctx:
        r = ctx.pipe_rates()
        assert r.sm_count > 0 and 500.0 < r.sm_clock_mhz < 3000.0
        for v in (r.ffma_per_clk_sm, r.ex2_per_clk_sm, r.lg2_per_clk_sm, r.fmnmx_per_clk_sm,
                  r.dfma_per_clk_sm):
            assert 0.0 < v <= 512.0
        assert r.lg2_per_clk_sm <= r.ffma_per_clk_sm and r.dfma_per_clk_sm <= r.ffma_per_clk_sm
