"""The tensor-core product the split-precision DFT is built on, against an
FP64 product: TF32 alone and the three-term TF32 split."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("terms,bound", [(1, 2.0 ** -9), (3, 2.0 ** -19)])
def test_tc_tile_product(terms, bound):
    import torch
    rng = np.random.default_rng(31 + terms)
    a = rng.standard_normal((128, 32)).astype(np.float32)
    b = rng.standard_normal((32, 32)).astype(np.float32)
    ref = a.astype(np.float64) @ b.astype(np.float64)
    at = torch.from_numpy(a).cuda()
    btt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    dt = torch.zeros((128, 32), dtype=torch.float32, device="cuda")
    t.tfft_tc_selftest(at, btt, dt, terms)
    d = dt.cpu().numpy().astype(np.float64)
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64)
    assert np.max(np.abs(d - ref) / scale) <= bound


def test_tc_tile_identity_and_permutation():
    """Exact small integers pass unchanged; a permutation matrix permutes."""
    import torch
    a = (np.arange(128 * 32) % 29 - 14).astype(np.float32).reshape(128, 32)
    perm = np.roll(np.eye(32, dtype=np.float32), 5, axis=1)
    at = torch.from_numpy(a).cuda()
    btt = torch.from_numpy(np.ascontiguousarray(perm.T)).cuda()
    dt = torch.zeros((128, 32), dtype=torch.float32, device="cuda")
    t.tfft_tc_selftest(at, btt, dt, 1)
    assert np.array_equal(dt.cpu().numpy(), a @ perm)
