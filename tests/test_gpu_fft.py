"""Parity of the CUDA transform with the FP64 oracle (no faults)."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import normal_batch, uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("abft", [False, True])
@pytest.mark.parametrize("log2n", list(range(0, 13)))
def test_single_pass_c64_all_sizes(log2n, abft):
    n = 1 << log2n
    batch = 37 if n >= 64 else 301          # several tiles and a ragged tail
    x = uniform_batch(n, batch, seed=100 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=abft)
    assert t.tfft_plan_info(plan)["passes"] == 1
    err = rel_err_rows(y, oracle_fft(x))
    assert err.max() <= tol(n, t.TFFT_C64), err.max()
    if abft:
        assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("abft", [False, True])
@pytest.mark.parametrize("log2n", [13, 14, 15, 16, 17, 18, 19, 20])
def test_multi_pass_c64(log2n, abft):
    n = 1 << log2n
    batch = max(3, (1 << 21) // n) + 1
    x = uniform_batch(n, batch, seed=200 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=abft)
    assert t.tfft_plan_info(plan)["passes"] >= 2
    err = rel_err_rows(y, oracle_fft(x))
    assert err.max() <= tol(n, t.TFFT_C64), err.max()
    if abft:
        assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n,passes", [(6, 2), (10, 2), (12, 2), (9, 3), (12, 3), (15, 3)])
def test_forced_pass_counts_agree(log2n, passes):
    n = 1 << log2n
    x = uniform_batch(n, 19, seed=300 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=True, force_passes=passes)
    assert t.tfft_plan_info(plan)["passes"] == passes
    err = rel_err_rows(y, oracle_fft(x))
    assert err.max() <= tol(n, t.TFFT_C64), err.max()
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [0, 1, 3, 6, 10, 11, 12, 14, 16, 20])
def test_c128(log2n):
    n = 1 << log2n
    batch = max(2, min(64, (1 << 20) // n)) + 1
    x = normal_batch(n, batch, seed=3)
    y, plan = run_gpu(x, t.TFFT_C128, abft=True)
    err = rel_err_rows(y, oracle_fft(x))
    assert err.max() <= tol(n, t.TFFT_C128), err.max()
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


def test_batch_one_and_group_larger_than_batch():
    for n in (16, 1024, 1 << 15):
        x = uniform_batch(n, 1, seed=7)
        y, plan = run_gpu(x, t.TFFT_C64, abft=True)
        assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
        t.tfft_destroy(plan)


def test_rejects_inplace_with_abft_and_bad_pointers():
    import torch
    x = torch.zeros(4, 64, dtype=torch.complex64, device="cuda")
    plan = t.tfft_plan(64, 4, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    with pytest.raises(t.TfftError) as e:
        t.tfft_exec(plan, x, x)
    assert e.value.code == -4
    with pytest.raises(t.TfftError):
        t.tfft_exec(plan, x.data_ptr() + 8, x)
    t.tfft_destroy(plan)
    plan = t.tfft_plan(64, 4, t.TFFT_C64, t.TFFT_ABFT_OFF)
    y = x.clone()
    t.tfft_exec(plan, y, y)          # in place is fine without ABFT
    torch.cuda.synchronize()
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [8, 16, 24])
def test_full_size_sampled_parity(log2n):
    """The 2^28-element (2 GiB) batch of the throughput sweep, in the bench's
    configuration (ABFT on), checked on sampled signals against the oracle."""
    import torch
    n = 1 << log2n
    batch = (1 << 28) // n
    xt = torch.from_numpy(uniform_batch(n, batch, seed=log2n)).cuda()
    yt = torch.empty_like(xt)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    t.tfft_exec(plan, xt, yt, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert t.tfft_report(plan) == (0, 0)
    rows = sorted({0, batch - 1, batch // 2, (batch * 7) // 11})
    x = xt[rows].cpu().numpy()
    y = yt[rows].cpu().numpy()
    err = rel_err_rows(y, oracle_fft(x))
    assert err.max() <= tol(n, t.TFFT_C64), err.max()
    t.tfft_destroy(plan)
    del xt, yt
    torch.cuda.empty_cache()


def test_c128_4096_one_pass_radix16():
    """complex128 N = 4096 runs as one pass of three radix-16 stages (one line
    a 256-thread tile): parity with the oracle over a batch with a ragged last
    group, the same output as the forced two-pass plan within tolerance, and
    a scaled value at every stage (input read, each radix stage) detected,
    named and corrected -- the correction recomputes through the direct-load
    pass kernel of the same radix."""
    n, batch = 4096, 37
    x = normal_batch(n, batch, seed=41)
    ref = oracle_fft(x)
    plan = t.tfft_plan(n, batch, t.TFFT_C128, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    assert info["passes"] == 1 and info["stages"][0] == 3 and info["tile_threads"][0] == 256
    y, _ = run_gpu(x, t.TFFT_C128, plan=plan)
    assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C128)
    assert t.tfft_report(plan) == (0, 0)
    y2, p2 = run_gpu(x, t.TFFT_C128, force_passes=2)
    assert t.tfft_plan_info(p2)["passes"] == 2
    assert rel_err_rows(y2, ref).max() <= tol(n, t.TFFT_C128)
    t.tfft_destroy(p2)
    rng = np.random.default_rng(43)
    for k, stage in enumerate((-1, 0, 1, 2)):
        sig, idx = int(rng.integers(batch)), int(rng.integers(n))
        fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=0, stage=stage, signal=sig, line=0, index=idx,
                     factor=1.0 + 1e-3)
        yf, _ = run_gpu(x, t.TFFT_C128, plan=plan, fault=fault)
        assert rel_err_rows(yf, ref).max() <= tol(n, t.TFFT_C128), stage
        assert t.tfft_report(plan) == (k + 1, k + 1), stage
        ev, _ = t.tfft_fault_log(plan)
        assert ev[-1]["signal"] == sig, stage
    t.tfft_destroy(plan)
