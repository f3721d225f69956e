"""Verification of few large groups by several blocks per group (their sums
meet in per-group accumulators, the last block decides and restores them):
clean execs stay clean, a fault is detected, located and corrected, and the
execs after it are clean again (Section III-A detection, III-B correction)."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("log2n,batch", [(21, 16), (20, 40)])
def test_split_verify_clean_fault_clean(log2n, batch):
    import torch
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=3100 + log2n)
    ref = oracle_fft(x)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    s = torch.cuda.current_stream()
    for _ in range(3):
        t.tfft_exec(plan, xt, yt, s)
    torch.cuda.synchronize()
    assert rel_err_rows(yt.cpu().numpy(), ref).max() <= tol(n, t.TFFT_C64)
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 0 and 0 < st["max_clean_ratio"] < 1.0
    p = info["passes"] - 1
    sig = batch - 3
    t.tfft_set_fault(plan, mode=t.TFFT_FAULT_SCALE, pass_=p, stage=0, signal=sig, line=5, index=3, factor=1.5)
    t.tfft_exec(plan, xt, yt, s)
    torch.cuda.synchronize()
    assert rel_err_rows(yt.cpu().numpy(), ref).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    ev, total = t.tfft_fault_log(plan)
    assert total == 1 and ev[0]["signal"] == sig
    for _ in range(2):
        t.tfft_exec(plan, xt, yt, s)
    torch.cuda.synchronize()
    assert rel_err_rows(yt.cpu().numpy(), ref).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n,batch,group,mode", [
    (8, 512, 64, t.TFFT_ABFT_TWO_SIDED),     # four groups in a verification block
    (8, 300, 7, t.TFFT_ABFT_TWO_SIDED),      # a group size that is no power of two, a short last group
    (10, 96, 0, t.TFFT_ABFT_ONE_SIDED),      # every signal its own group
    (16, 70, 64, t.TFFT_ABFT_TWO_SIDED),     # one group per block, its signals in rounds
    (13, 100, 16, t.TFFT_ABFT_TWO_SIDED),    # sixteen lanes per signal
])
def test_verification_layouts_clean_and_one_fault(log2n, batch, group, mode):
    """Whatever the block layout of the verification (groups per block,
    lanes per signal, rounds), clean execs are clean and a value added to
    one input element is detected, named and corrected."""
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=3300 + log2n + group)
    ref = oracle_fft(x)
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, mode, group=group)
    try:
        y, _ = run_gpu(x, t.TFFT_C64, plan=plan)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
        assert t.tfft_report(plan) == (0, 0)
        info = t.tfft_plan_info(plan)
        sig = batch - 2
        fault = dict(mode=t.TFFT_FAULT_ADD, pass_=0, stage=-1, signal=sig,
                     line=min(3, info["lines_per_signal"][0] - 1), index=5, factor=100.0)
        y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
        assert t.tfft_report(plan) == (1, 1)
        ev, _ = t.tfft_fault_log(plan)
        assert ev[-1]["signal"] == sig
        t.tfft_set_fault(plan, mode=t.TFFT_FAULT_NONE)
        y, _ = run_gpu(x, t.TFFT_C64, plan=plan)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
        assert t.tfft_report(plan) == (1, 1)
    finally:
        t.tfft_destroy(plan)
