"""Fault-coverage and false-alarm campaigns on the GPU (Section II-A fault
model: one flipped bit of one value, at a random pass, stage, signal, line,
element and bit).  A fault is harmful when the uncorrected output of its
signal misses the tolerance against the FP64 oracle; every harmful fault must
be detected, attributed to its signal and corrected, and every other output
must stay within the tolerance."""
import pytest

import paper_2405_02520_gb300 as t
from tests.campaign import clean_campaign, run_campaign

pytestmark = pytest.mark.gpu

CAMPAIGNS = [(8, 64, t.TFFT_C64), (10, 64, t.TFFT_C64), (12, 32, t.TFFT_C64), (13, 32, t.TFFT_C64),
             (16, 8, t.TFFT_C64), (18, 4, t.TFFT_C64), (19, 4, t.TFFT_C64), (20, 4, t.TFFT_C64),
             (21, 2, t.TFFT_C64), (22, 2, t.TFFT_C64), (24, 1, t.TFFT_C64),
             (12, 32, t.TFFT_C128), (20, 64, t.TFFT_C128)]


@pytest.mark.parametrize("log2n,batch,dtype", CAMPAIGNS)
def test_every_harmful_bitflip_detected_located_and_corrected(log2n, batch, dtype):
    """60 random bit flips: harmful ones (including those within a factor of
    two of the tolerance) are all detected, named and corrected; benign ones
    leave every output within the tolerance.  Complex128 2^20 x 64 is the
    one-fault-per-launch configuration, corrected to 1e-14 log2 N."""
    r = run_campaign(1 << log2n, batch, dtype, faults=60, seed=log2n)
    assert r["harmful"] > 0 and r["clear"] > 0
    assert r["harmful_detected"] == r["harmful"], r
    assert r["harmful_located"] == r["harmful"], r
    assert r["harmful_corrected"] == r["harmful"], r
    assert r["benign_output_ok"] == r["benign"], r


def test_config1_ten_thousand_clean_launches_no_false_positive():
    r = clean_campaign(1024, 256, 10000)
    assert r["detected"] == 0, r


def test_n8192_ten_thousand_clean_launches_no_false_positive():
    """N = 2^13, the length whose clean residuals came closest to the
    threshold over the 2^28-element sweep."""
    r = clean_campaign(1 << 13, 256, 10000)
    assert r["detected"] == 0, r


def test_large_n_ten_thousand_clean_launches_no_false_positive():
    r = clean_campaign(1 << 16, 64, 10000)
    assert r["detected"] == 0, r
