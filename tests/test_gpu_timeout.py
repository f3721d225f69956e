"""The bounded tile-copy waits give up, report a timeout and leave the device
usable.  A plan whose waits may not poll at all (wait_polls = -1) makes every
wait for a tile copy give up at once: the kernels set the plan's error flag,
drain the copies already in flight and return; tfft_report then raises
TFFT_ERR_TIMEOUT.  Nothing faults or hangs: the waits end by themselves.
Afterwards the same device runs correct transforms, and a reset clears the
recorded timeout."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import np_dtype, oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu

TIMEOUT = -7


@pytest.mark.parametrize("log2n,batch,dtype", [(6, 64, t.TFFT_C64),      # legacy TMA tile kernel
                                               (10, 64, t.TFFT_C64),     # single-pass tile kernel
                                               (14, 32, t.TFFT_C64),     # two passes
                                               (21, 2, t.TFFT_C64),      # three passes
                                               (12, 16, t.TFFT_C128)])
def test_wait_that_cannot_poll_reports_timeout_then_device_recovers(log2n, batch, dtype):
    import torch
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=77).astype(np_dtype(dtype))
    plan = t.tfft_plan_ex(n, batch, dtype, t.TFFT_ABFT_TWO_SIDED, wait_polls=-1)
    try:
        xt = torch.from_numpy(x).cuda()
        yt = torch.empty_like(xt)
        t.tfft_exec(plan, xt, yt, torch.cuda.current_stream())
        torch.cuda.synchronize()
        with pytest.raises(t.TfftError) as e:
            t.tfft_report(plan)
        assert e.value.code == TIMEOUT
        # the flag stays until a reset clears it
        with pytest.raises(t.TfftError):
            t.tfft_report_ex(plan)
        t.tfft_reset_counters(plan)
        assert t.tfft_report(plan) == (0, 0)
    finally:
        t.tfft_destroy(plan)
    # the device still runs correct transforms
    y, p2 = run_gpu(x, dtype)
    try:
        assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, dtype)
        assert t.tfft_report(p2) == (0, 0)
    finally:
        t.tfft_destroy(p2)


def test_default_and_explicit_poll_limits_run_clean():
    """wait_polls = 0 (default) and a generous explicit limit give the same
    correct result as each other."""
    n, batch = 1 << 12, 32
    x = uniform_batch(n, batch, seed=78)
    ya, pa = run_gpu(x, t.TFFT_C64)
    yb, pb = run_gpu(x, t.TFFT_C64, wait_polls=1 << 22)
    try:
        assert np.array_equal(ya, yb)
        assert rel_err_rows(ya, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
        assert t.tfft_report(pb) == (0, 0)
    finally:
        t.tfft_destroy(pa)
        t.tfft_destroy(pb)
