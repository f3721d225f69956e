"""Inverse and normalised transforms on the GPU (Section II: the inverse DFT
x_j = (1/N) sum_n y_n e^{+2 pi i jn/N}) against the FP64 oracle, with the
two-sided checksums still detecting and correcting a fault."""
import numpy as np
import pytest

import oracle
import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import normal_batch, uniform_batch
from tests.gpu_util import rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


def _ifft(x):
    return oracle.ifft(x.astype(np.complex128))


@pytest.mark.parametrize("log2n", [1, 4, 8, 10, 12, 13, 16, 19])
def test_inverse_normalised_c64(log2n):
    n = 1 << log2n
    batch = max(3, (1 << 20) // n) + 1
    x = uniform_batch(n, batch, seed=500 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=True, direction=t.TFFT_INVERSE, normalize=True)
    info = t.tfft_plan_info(plan)
    assert info["direction"] == t.TFFT_INVERSE and info["normalize"] == 1
    assert rel_err_rows(y, _ifft(x)).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [6, 11, 15])
def test_inverse_unnormalised_and_forward_normalised(log2n):
    n = 1 << log2n
    x = uniform_batch(n, 37, seed=600 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=True, direction=t.TFFT_INVERSE)
    assert rel_err_rows(y, n * _ifft(x)).max() <= tol(n, t.TFFT_C64)
    t.tfft_destroy(plan)
    y, plan = run_gpu(x, t.TFFT_C64, abft=True, normalize=True)
    assert rel_err_rows(y, oracle.fft(x.astype(np.complex128)) / n).max() <= tol(n, t.TFFT_C64)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [9, 12, 20])
def test_inverse_c128(log2n):
    n = 1 << log2n
    x = normal_batch(n, 5, seed=700 + log2n, dtype=np.complex128)
    y, plan = run_gpu(x, t.TFFT_C128, abft=True, direction=t.TFFT_INVERSE, normalize=True)
    assert rel_err_rows(y, _ifft(x)).max() <= tol(n, t.TFFT_C128)
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [10, 16])
def test_round_trip(log2n):
    """forward, then the normalised inverse, gives the input back."""
    import torch
    n = 1 << log2n
    x = uniform_batch(n, 64, seed=800 + log2n)
    xt = torch.from_numpy(x).cuda()
    yt, zt = torch.empty_like(xt), torch.empty_like(xt)
    fwd = t.tfft_plan_ex(n, 64, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    inv = t.tfft_plan_ex(n, 64, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, direction=t.TFFT_INVERSE, normalize=True)
    t.tfft_exec(fwd, xt, yt, torch.cuda.current_stream())
    t.tfft_exec(inv, yt, zt, torch.cuda.current_stream())
    torch.cuda.synchronize()
    z = zt.cpu().numpy()
    assert rel_err_rows(z, x.astype(np.complex128)).max() <= 2 * tol(n, t.TFFT_C64)
    assert t.tfft_report(fwd) == (0, 0) and t.tfft_report(inv) == (0, 0)
    t.tfft_destroy(fwd)
    t.tfft_destroy(inv)


@pytest.mark.parametrize("log2n,stage_from_end", [(10, 1), (14, 1), (20, 2)])
def test_inverse_fault_detected_located_corrected(log2n, stage_from_end):
    """A scaled intermediate value in the inverse transform is caught by the
    checksums of the underlying forward transform and corrected."""
    n = 1 << log2n
    batch = 48
    x = uniform_batch(n, batch, seed=900 + log2n)
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, direction=t.TFFT_INVERSE,
                          normalize=True)
    info = t.tfft_plan_info(plan)
    p = info["passes"] - 1
    sig = 21
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=p, stage=max(-1, info["stages"][p] - stage_from_end),
                 signal=sig, line=0, index=5, factor=1.5)
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    ref = _ifft(x)
    assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    ev, total = t.tfft_fault_log(plan)
    assert total == 1 and ev[0]["signal"] == sig
    t.tfft_destroy(plan)
