"""tfft_exec_host: host buffers in and out, the batch cut into chunks of
whole checksum groups whose copies overlap the transforms; the result equals
the device-buffer exec bit for bit, the checksums stay clean, an armed fault
(one chunk) is corrected, and the fault log names the signal of the batch."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, tol

pytestmark = pytest.mark.gpu


def _pinned(x):
    import torch
    h = torch.empty(x.shape, dtype=torch.complex64, pin_memory=True)
    h.copy_(torch.from_numpy(x))
    return h


@pytest.mark.parametrize("log2n,batch", [(10, 16), (10, 200), (12, 37), (16, 300), (20, 40), (8, 4099)])
def test_exec_host_matches_device_exec(log2n, batch):
    import torch
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=4100 + log2n)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    hin, hout = _pinned(x), torch.empty((batch, n), dtype=torch.complex64, pin_memory=True)
    s = torch.cuda.current_stream()
    for _ in range(2):                       # the second call reuses streams, events and staging
        hout.zero_()
        t.tfft_exec_host(plan, hin, hout, s)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    t.tfft_exec(plan, xd, yd, s)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy(), yd.cpu().numpy())
    if n * batch <= (1 << 22):
        assert rel_err_rows(hout.numpy(), oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 0 and st["execs"] == 3
    t.tfft_destroy(plan)


def test_exec_host_armed_fault_corrected():
    import torch
    n, batch = 4096, 96
    x = uniform_batch(n, batch, seed=4200)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    hin, hout = _pinned(x), torch.empty((batch, n), dtype=torch.complex64, pin_memory=True)
    sig = 77                                  # in the fifth group of sixteen
    t.tfft_set_fault(plan, mode=t.TFFT_FAULT_SCALE, pass_=0, stage=info["stages"][0] - 1, signal=sig,
                     line=0, index=9, factor=1.5)
    t.tfft_exec_host(plan, hin, hout, torch.cuda.current_stream())
    assert rel_err_rows(hout.numpy(), oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    ev, total = t.tfft_fault_log(plan)
    assert total == 1 and ev[0]["signal"] == sig and ev[0]["group"] == sig // 16
    t.tfft_destroy(plan)


@pytest.mark.parametrize("mode,dtype,precision", [(t.TFFT_ABFT_ONE_SIDED, t.TFFT_C64, t.TFFT_PREC_FP32),
                                                  (t.TFFT_ABFT_TWO_SIDED, t.TFFT_C128, t.TFFT_PREC_FP32),
                                                  (t.TFFT_ABFT_TWO_SIDED, t.TFFT_C64, t.TFFT_PREC_BF16X3),
                                                  (t.TFFT_ABFT_OFF, t.TFFT_C64, t.TFFT_PREC_FP32)])
def test_exec_host_other_modes_match_device_exec(mode, dtype, precision):
    import torch
    n, batch = 4096, 150
    x = uniform_batch(n, batch, seed=4300, dtype=np.complex128 if dtype == t.TFFT_C128 else np.complex64)
    plan = t.tfft_plan_ex(n, batch, dtype, mode, precision=precision)
    tdt = torch.complex128 if dtype == t.TFFT_C128 else torch.complex64
    hin = torch.empty((batch, n), dtype=tdt, pin_memory=True)
    hin.copy_(torch.from_numpy(x))
    hout = torch.empty_like(hin)
    s = torch.cuda.current_stream()
    t.tfft_exec_host(plan, hin, hout, s)
    xd = hin.cuda()
    yd = torch.empty_like(xd)
    t.tfft_exec(plan, xd, yd, s)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy(), yd.cpu().numpy())
    assert t.tfft_report(plan)[0] == 0
    t.tfft_destroy(plan)
