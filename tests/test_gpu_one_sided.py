"""One-sided ABFT mode (Section III: the left-side checksum of each signal
alone; a flagged signal is recomputed) on the GPU."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


def _plan(n, batch, dtype=t.TFFT_C64, **kw):
    return t.tfft_plan_ex(n, batch, dtype, t.TFFT_ABFT_ONE_SIDED, **kw)


@pytest.mark.parametrize("log2n", [8, 10, 12, 13, 16, 20])
def test_one_sided_clean(log2n):
    n = 1 << log2n
    batch = max(2, (1 << 20) // n) + 3
    x = uniform_batch(n, batch, seed=1100 + log2n)
    plan = _plan(n, batch)
    info = t.tfft_plan_info(plan)
    assert info["abft_mode"] == t.TFFT_ABFT_ONE_SIDED
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan)
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 0 and st["max_clean_ratio"] < 1.0
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [8, 11, 14, 19])
def test_one_sided_fault_named_and_recomputed(log2n):
    """The faulty signal is named by its own checksum; its output is
    recomputed from the input."""
    n = 1 << log2n
    batch = 40
    x = uniform_batch(n, batch, seed=1200 + log2n)
    plan = _plan(n, batch)
    info = t.tfft_plan_info(plan)
    p = info["passes"] - 1
    sig = 29
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=p, stage=info["stages"][p] - 1, signal=sig, line=0,
                 index=3, factor=1.25)
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    ev, total = t.tfft_fault_log(plan)
    assert total == 1 and ev[0]["signal"] == sig and ev[0]["group"] == sig
    t.tfft_destroy(plan)


def test_one_sided_unsupported_below_the_tile_kernels():
    with pytest.raises(t.TfftError) as e:
        _plan(64, 16)
    assert e.value.code == -2


def test_one_sided_c128():
    n = 1 << 12
    x = uniform_batch(n, 9, seed=1300, dtype=np.complex128)
    plan = _plan(n, 9, t.TFFT_C128)
    y, _ = run_gpu(x, t.TFFT_C128, plan=plan)
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C128)
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)
