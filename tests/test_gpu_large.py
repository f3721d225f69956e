"""Transforms longer than 2^26 (three passes with 1024-point sub-transforms),
checked on sampled outputs against the oracle's definition sum, by Parseval,
and with a corrected fault."""
import numpy as np
import pytest

import oracle
import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import tol

pytestmark = pytest.mark.gpu


def _run(n, batch, fault=None):
    import torch
    x = uniform_batch(n, batch, seed=1400 + int(np.log2(n)))
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    if fault is not None:
        t.tfft_set_fault(plan, **fault)
    t.tfft_exec(plan, xt, yt, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return x, yt.cpu().numpy(), plan


def _check_bins(x, y, n, nbins, seed):
    rng = np.random.default_rng(seed)
    ks = [0, n - 1] + rng.integers(0, n, size=nbins).tolist()
    ref = oracle.dft_bins(x, ks)
    # per-output bound: the relative-L2 tolerance times the RMS output size
    scale = np.sqrt(n) * np.linalg.norm(x.astype(np.complex128))
    err = np.abs(y[ks].astype(np.complex128) - ref)
    assert err.max() <= 8 * tol(n, t.TFFT_C64) * scale / np.sqrt(n), (err.max(), scale)


@pytest.mark.parametrize("log2n", [27, 28])
def test_long_transform_sampled_bins_and_parseval(log2n):
    n = 1 << log2n
    x, y, plan = _run(n, 1)
    info = t.tfft_plan_info(plan)
    assert info["passes"] == 3 and max(info["nsub"]) <= 1024
    _check_bins(x[0], y[0], n, 4, seed=log2n)
    ex = np.sum(np.abs(x[0].astype(np.complex128)) ** 2)
    ey = np.sum(np.abs(y[0].astype(np.complex128)) ** 2)
    assert abs(ey / (n * ex) - 1) <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


def test_long_transform_fault_corrected():
    n = 1 << 27
    plan0 = t.tfft_plan(n, 2, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan0)
    t.tfft_destroy(plan0)
    # an intermediate value of the middle pass scaled by 10^4: harmful (a 1 %
    # change of one intermediate value of a 2^27-point transform is below
    # the rounding-level threshold and leaves the output within tolerance)
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=1, stage=info["stages"][1] - 1, signal=1, line=3,
                 index=7, factor=1e4)
    x, y, plan = _run(n, 2, fault)
    assert t.tfft_report(plan) == (1, 1)
    _check_bins(x[1], y[1], n, 3, seed=99)
    t.tfft_destroy(plan)
