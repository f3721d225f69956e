"""Split-precision DFT on the tensor cores (radix-16 butterflies as dense
products) against the FP64 oracle: error per form, tones far below the
largest, checksums without false alarms, a corrected fault."""
import numpy as np
import pytest

import oracle
import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu

# relative-L2 bound per signal, in units of the complex64 tolerance
# 2e-6 log2 N: the two three-term split forms keep about 21 (TF32) and 16
# (BF16) significant bits and are held to the complex64 tolerance itself;
# plain TF32 (10 stored bits, unit roundoff 2^-11) is held to 64 times it.
FORM_BOUND = {t.TFFT_PREC_TF32X3: 1.0, t.TFFT_PREC_BF16X3: 1.0, t.TFFT_PREC_TF32: 64.0}


@pytest.mark.parametrize("precision", [t.TFFT_PREC_TF32X3, t.TFFT_PREC_BF16X3, t.TFFT_PREC_TF32])
@pytest.mark.parametrize("log2n", [8, 9, 10, 11, 12, 16])
def test_tc_forms_match_oracle(log2n, precision):
    n = 1 << log2n
    batch = max(2, (1 << 20) // n) + 1
    x = uniform_batch(n, batch, seed=1500 + log2n)
    y, plan = run_gpu(x, t.TFFT_C64, abft=True, precision=precision)
    info = t.tfft_plan_info(plan)
    assert info["precision"] == precision
    err = rel_err_rows(y, oracle_fft(x)).max()
    assert err <= FORM_BOUND[precision] * tol(n, t.TFFT_C64), err
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 0 and st["max_clean_ratio"] < 1.0
    t.tfft_destroy(plan)


def _tones(n, batch, seed):
    """8 tones per signal, bins uniform, amplitudes 10^U[-3,0], phases U[0,2pi),
    plus complex Gaussian noise of standard deviation 1e-4 per component."""
    rng = np.random.default_rng(seed)
    k = np.arange(n)
    x = np.zeros((batch, n), dtype=np.complex128)
    bins = rng.integers(0, n, size=(batch, 8))
    amp = 10.0 ** rng.uniform(-3, 0, size=(batch, 8))
    ph = rng.uniform(0, 2 * np.pi, size=(batch, 8))
    for b in range(batch):
        for q in range(8):
            x[b] += amp[b, q] * np.exp(1j * (2 * np.pi * bins[b, q] * k / n + ph[b, q]))
    x += 1e-4 * (rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n)))
    return x.astype(np.complex64), bins, amp


@pytest.mark.parametrize("log2n", [12, 16])
def test_tc_split_keeps_small_tones(log2n):
    """The smallest tones (amplitude down to 1e-3 of the largest) come out of
    the split-TF32 form with the accuracy of the complex64 path."""
    n = 1 << log2n
    x, bins, amp = _tones(n, 6, seed=4)
    ref = oracle_fft(x)
    y32, p32 = run_gpu(x, t.TFFT_C64, abft=True)
    ytc, ptc = run_gpu(x, t.TFFT_C64, abft=True, precision=t.TFFT_PREC_TF32X3)
    for b in range(x.shape[0]):
        q = int(np.argmin(amp[b]))
        k = bins[b, q]
        e32 = abs(y32[b, k] - ref[b, k]) / abs(ref[b, k])
        etc = abs(ytc[b, k] - ref[b, k]) / abs(ref[b, k])
        assert etc <= max(16 * e32, 1e-4), (b, amp[b, q], e32, etc)
    t.tfft_destroy(p32)
    t.tfft_destroy(ptc)


@pytest.mark.parametrize("precision", [t.TFFT_PREC_TF32X3, t.TFFT_PREC_BF16X3])
def test_tc_fault_detected_and_corrected(precision):
    n, batch = 4096, 64
    x = uniform_batch(n, batch, seed=1600)
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, precision=precision)
    info = t.tfft_plan_info(plan)
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=0, stage=info["stages"][0] - 1, signal=37, line=0, index=100,
                 factor=1.5)
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    assert rel_err_rows(y, oracle_fft(x)).max() <= FORM_BOUND[precision] * tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    t.tfft_destroy(plan)


def test_tc_unsupported_lengths():
    with pytest.raises(t.TfftError) as e:
        t.tfft_plan_ex(1 << 13, 4, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, precision=t.TFFT_PREC_TF32X3)
    assert e.value.code == -2
    with pytest.raises(t.TfftError) as e:
        t.tfft_plan_ex(1 << 10, 4, t.TFFT_C128, t.TFFT_ABFT_TWO_SIDED, precision=t.TFFT_PREC_TF32X3)
    assert e.value.code == -2
    with pytest.raises(t.TfftError) as e:
        t.tfft_plan_ex(1 << 14, 4, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, precision=t.TFFT_PREC_BF16X3)
    assert e.value.code == -2
