"""The allocation-free entry point tfft_exec_noalloc, called through the C ABI,
against the plan-based tfft_exec on the same inputs, two calls in a row.

It serves callers that may not allocate device memory (graph captures that
must not hold allocation nodes, externally managed memory, real-time loops).
This file is collected last so that a failure here cannot hide another test.
"""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.astype(np.complex128); b = b.astype(np.complex128)
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("log2n,batch", [(13, 37), (16, 9), (18, 32)])
def test_noalloc_matches_plan_exec_twice(log2n, batch):
    import torch
    n = 1 << log2n
    tolerance = 2e-6 * log2n
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_OFF)
    try:
        for call in range(2):
            x = torch.from_numpy(uniform_batch(n, batch, seed=500 + 10 * log2n + call)).cuda()
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            t.tfft_exec(plan, x, y_ref, torch.cuda.current_stream())
            t.tfft_exec_noalloc(n, batch, x, y, torch.cuda.current_stream())
            torch.cuda.synchronize()
            err = _rel(y.cpu().numpy(), y_ref.cpu().numpy())
            assert np.all(np.isfinite(err)) and err.max() <= tolerance, (call, err.max())
    finally:
        t.tfft_destroy(plan)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda")
    for n, batch in (((1 << 13), (1 << 23) // (1 << 13) + 1), (4096, 1), ((1 << 19), 1), (12288, 1)):
        with pytest.raises(t.TfftError) as e:
            t.tfft_exec_noalloc(n, batch, x, x)
        assert e.value.code == -1
