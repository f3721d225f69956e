"""The allocation-free entry point tfft_exec_noalloc, called through the C ABI.

It serves callers that may not allocate device memory (code under a memory
manager or sandbox that owns every device allocation, real-time loops that may
not block on the allocator).  Its output is checked against the FP64 oracle
and against the plan-based tfft_exec on the same inputs, two calls in a row.
This file is collected last so that a failure here cannot hide another test.
"""
import numpy as np
import pytest

import oracle
import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.astype(np.complex128); b = b.astype(np.complex128)
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def test_noalloc_setup_only_call():
    """n = 0, batch = 0 performs only the per-device set-up and succeeds."""
    t.tfft_exec_noalloc(0, 0, 0, 0)
    t.tfft_exec_noalloc(0, 0, 0, 0)


@pytest.mark.parametrize("log2n,batch", [(13, 37), (16, 9), (18, 32)])
def test_noalloc_matches_oracle_and_plan_exec_twice(log2n, batch):
    import torch
    n = 1 << log2n
    tolerance = 2e-6 * log2n
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_OFF)
    try:
        for call in range(2):
            xh = uniform_batch(n, batch, seed=500 + 10 * log2n + call)
            x = torch.from_numpy(xh).cuda()
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            t.tfft_exec(plan, x, y_ref, torch.cuda.current_stream())
            t.tfft_exec_noalloc(n, batch, x, y, torch.cuda.current_stream())
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            e_plan = _rel(yh, y_ref.cpu().numpy())
            e_oracle = _rel(yh, oracle.fft(xh.astype(np.complex128)))
            assert np.all(np.isfinite(e_plan)) and e_plan.max() <= tolerance, (call, e_plan.max())
            assert np.all(np.isfinite(e_oracle)) and e_oracle.max() <= tolerance, (call, e_oracle.max())
    finally:
        t.tfft_destroy(plan)


def test_noalloc_in_place_twice():
    """in == out: the first pass reads the input before the second writes."""
    import torch
    n, batch = 1 << 15, 24
    for call in range(2):
        xh = uniform_batch(n, batch, seed=900 + call)
        x = torch.from_numpy(xh).cuda()
        t.tfft_exec_noalloc(n, batch, x, x, torch.cuda.current_stream())
        torch.cuda.synchronize()
        err = _rel(x.cpu().numpy(), oracle.fft(xh.astype(np.complex128)))
        assert err.max() <= 2e-6 * 15, (call, err.max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    for n, batch in (((1 << 13), (1 << 23) // (1 << 13) + 1), (4096, 1), ((1 << 19), 1), (12288, 1),
                     (0, 1), ((1 << 13), 0)):
        with pytest.raises(t.TfftError) as e:
            t.tfft_exec_noalloc(n, batch, x, x)
        assert e.value.code == -1
