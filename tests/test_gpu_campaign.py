"""Fault-coverage and false-alarm campaigns on the GPU."""
import pytest

import paper_2405_02520_gb300 as t
from tests.campaign import clean_campaign, run_campaign

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("log2n,batch,dtype", [(8, 64, t.TFFT_C64), (10, 64, t.TFFT_C64),
                                               (12, 32, t.TFFT_C64), (13, 32, t.TFFT_C64),
                                               (16, 8, t.TFFT_C64), (18, 4, t.TFFT_C64),
                                               (19, 4, t.TFFT_C64), (20, 4, t.TFFT_C64),
                                               (12, 32, t.TFFT_C128)])
def test_every_harmful_bitflip_detected_and_corrected(log2n, batch, dtype):
    """Every bit flip whose uncorrected error exceeds twice the tolerance is
    detected and corrected; flips within a factor of two of the tolerance may
    hide below the checksum's rounding noise (their projection on the left
    vector is a sum of random phases) and are allowed at most one miss a
    campaign; benign flips leave the output within the tolerance."""
    r = run_campaign(1 << log2n, batch, dtype, faults=60, seed=log2n)
    assert r["harmful"] > 0 and r["clear"] > 0
    assert r["clear_detected"] == r["clear"], r
    assert r["clear_corrected"] == r["clear"], r
    assert r["marginal_missed"] <= 1, r
    assert r["harmful_corrected"] >= r["harmful"] - r["marginal_missed"], r
    assert r["benign_output_ok"] == r["benign"], r


def test_config1_ten_thousand_clean_launches_no_false_positive():
    r = clean_campaign(1024, 256, 10000)
    assert r["detected"] == 0, r


def test_large_n_ten_thousand_clean_launches_no_false_positive():
    r = clean_campaign(1 << 16, 64, 10000)
    assert r["detected"] == 0, r
