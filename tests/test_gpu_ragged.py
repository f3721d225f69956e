"""Ragged batches (signals of different lengths packed back to back) on the
GPU against the oracle, with graph replay, re-capture and corrected faults,
in the bucket-stream form and the persistent pass-family form."""
import numpy as np
import pytest

import oracle
import paper_2405_02520_gb300 as t
from tests.gpu_util import Guarded, rel_err_rows, tol

pytestmark = pytest.mark.gpu


def _ragged_input(count, seed, lo=6, hi=16):
    rng = np.random.default_rng(seed)
    lengths = (1 << rng.integers(lo, hi + 1, size=count)).astype(np.int64)
    total = int(lengths.sum())
    x = np.empty(total, dtype=np.complex64)
    x.real = rng.uniform(-1, 1, total).astype(np.float32)
    x.imag = rng.uniform(-1, 1, total).astype(np.float32)
    return lengths, x


def _check(lengths, x, y, *guarded):
    for g in guarded:
        g.check("ragged buffer")
    off = np.concatenate([[0], np.cumsum(lengths)])
    worst = 0.0
    for n in np.unique(lengths):
        idx = np.nonzero(lengths == n)[0]
        xs = np.stack([x[off[i]:off[i] + n] for i in idx])
        ys = np.stack([y[off[i]:off[i] + n] for i in idx])
        err = rel_err_rows(ys, oracle.fft(xs.astype(np.complex128))).max()
        assert err <= tol(int(n), t.TFFT_C64), (int(n), err)
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("autotune,staged,persistent", [(False, False, False), (True, False, False),
                                                        (False, True, False), (False, False, True),
                                                        (False, True, True)])
def test_ragged_matches_oracle_and_replays(autotune, staged, persistent):
    import torch
    lengths, x = _ragged_input(400, seed=5)
    r = t.Ragged(lengths.tolist(), autotune=autotune, staged=staged, persistent=persistent)
    fams, pb = r.families()
    if persistent:
        # every bucket of 256 points or more runs on the 256-thread tile kernels
        assert pb == sum(1 for n in set(lengths.tolist()) if n >= 256) and fams >= pb, (fams, pb)
    else:
        assert (fams, pb) == (0, 0)
    assert sorted(n for n, _ in r.info()) == sorted(set(lengths.tolist()))
    # lengths 2^6..2^16: every offset is a multiple of 64 elements, so every
    # bucket is addressed in place unless staging is forced
    assert all(d != staged for d in r.layout().values()), r.layout()
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    r.exec(xt, yt)                       # captured
    torch.cuda.synchronize()
    y1 = yt.cpu().numpy()
    _check(lengths, x, y1, xg, yg)
    yt.zero_()
    r.exec(xt, yt)                       # replayed
    torch.cuda.synchronize()
    assert np.array_equal(yt.cpu().numpy(), y1)
    y2g = Guarded(x.shape, xg.t.dtype)
    y2t = y2g.t
    r.exec(xt, y2t)                      # new output pointer: re-captured
    torch.cuda.synchronize()
    assert np.array_equal(y2t.cpu().numpy(), y1)
    st = r.report()
    assert st["detected"] == 0 and st["execs"] == 3
    r.destroy()


@pytest.mark.parametrize("persistent", [False, True])
def test_ragged_faults_in_two_buckets_corrected(persistent):
    import torch
    lengths, x = _ragged_input(300, seed=55)
    r = t.Ragged(lengths.tolist(), autotune=False, persistent=persistent)
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    r.exec(xt, yt)
    torch.cuda.synchronize()
    small = int(np.nonzero(lengths == 256)[0][3])
    large = int(np.nonzero(lengths == 1 << 15)[0][2])
    passes = dict(r.info())
    r.set_fault(small, mode=t.TFFT_FAULT_SCALE, pass_=0, stage=0, line=0, index=9, factor=2.0)
    r.set_fault(large, mode=t.TFFT_FAULT_SCALE, pass_=passes[1 << 15] - 1, stage=0, line=1, index=4,
                factor=2.0)
    r.exec(xt, yt)
    torch.cuda.synchronize()
    _check(lengths, x, yt.cpu().numpy(), xg, yg)
    st = r.report()
    assert st["detected"] == 2 and st["corrected"] + st["recomputed"] == 2
    r.destroy()


def _fault_sites(lengths, per_1000, seed):
    """Signals to fault, one per `1000 / per_1000` signals, in distinct ABFT
    groups (16 consecutive signals of one length), at most four per length
    and one per length below 256 points."""
    rng = np.random.default_rng(seed)
    want = max(1, len(lengths) * per_1000 // 1000)
    order = rng.permutation(len(lengths))
    local = {}
    counts = {}
    for i, n in enumerate(lengths):
        local[i] = counts.get(int(n), 0)
        counts[int(n)] = local[i] + 1
    used, per_len, out = set(), {}, []
    for i in order:
        n = int(lengths[i])
        g = (n, local[i] // 16)
        cap = 1 if n < 256 else 4
        if g in used or per_len.get(n, 0) >= cap:
            continue
        used.add(g)
        per_len[n] = per_len.get(n, 0) + 1
        out.append(int(i))
        if len(out) == want:
            break
    return out


@pytest.mark.parametrize("persistent", [False, True])
def test_ragged_one_fault_per_thousand_signals(persistent):
    """4000 signals (2^6..2^12 points), four faults in distinct groups in one
    exec: all detected and corrected."""
    import torch
    lengths, x = _ragged_input(4000, seed=505, lo=6, hi=12)
    r = t.Ragged(lengths.tolist(), autotune=False, persistent=persistent)
    passes = dict(r.info())
    sites = _fault_sites(lengths, 1, seed=7)
    assert len(sites) == 4
    for k, i in enumerate(sites):
        n = int(lengths[i])
        r.set_fault(i, mode=t.TFFT_FAULT_SCALE, pass_=passes[n] - 1, stage=0, line=0, index=(3 * k + 1) % n,
                    factor=3.0)
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    r.exec(xt, yt)
    torch.cuda.synchronize()
    _check(lengths, x, yt.cpu().numpy(), xg, yg)
    st = r.report()
    assert st["detected"] == 4 and st["corrected"] + st["recomputed"] == 4, st
    r.destroy()


@pytest.mark.parametrize("persistent", [False, True])
def test_ragged_mixed_direct_and_staged_buckets(persistent):
    """Lengths 2, 8, 256, 8192 and 65536: the short signals leave the
    multi-pass buckets' offsets off the 16-element box grid, so those buckets
    are staged while the others are addressed in place; faults in a staged and
    in a direct bucket are both corrected."""
    import torch
    rng = np.random.default_rng(77)
    lengths = rng.choice(np.array([2, 8, 256, 8192, 65536], dtype=np.int64), size=90)
    lengths[:2] = [2, 8192]             # make sure an 8192-point offset is misaligned
    total = int(lengths.sum())
    x = np.empty(total, dtype=np.complex64)
    x.real = rng.uniform(-1, 1, total).astype(np.float32)
    x.imag = rng.uniform(-1, 1, total).astype(np.float32)
    r = t.Ragged(lengths.tolist(), autotune=False, persistent=persistent)
    lay = r.layout()
    assert lay[8192] is False and lay[256] is True and lay[2] is True, lay
    passes = dict(r.info())
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    r.exec(xt, yt)
    torch.cuda.synchronize()
    _check(lengths, x, yt.cpu().numpy(), xg, yg)
    s8k = int(np.nonzero(lengths == 8192)[0][1])
    s256 = int(np.nonzero(lengths == 256)[0][2])
    r.set_fault(s8k, mode=t.TFFT_FAULT_SCALE, pass_=passes[8192] - 1, stage=0, line=0, index=3, factor=2.0)
    r.set_fault(s256, mode=t.TFFT_FAULT_SCALE, pass_=0, stage=0, line=0, index=5, factor=2.0)
    r.exec(xt, yt)
    torch.cuda.synchronize()
    _check(lengths, x, yt.cpu().numpy(), xg, yg)
    st = r.report()
    assert st["detected"] == 2 and st["corrected"] + st["recomputed"] == 2, st
    r.destroy()


@pytest.mark.parametrize("persistent", [False, True])
def test_ragged_one_sided_recompute_in_place(persistent):
    """One-sided checks on a ragged batch addressed in place: a detected
    signal is recomputed from the caller's input and written back at its
    caller offset."""
    import torch
    lengths, x = _ragged_input(120, seed=909, lo=8, hi=14)
    r = t.Ragged(lengths.tolist(), abft_mode=t.TFFT_ABFT_ONE_SIDED, autotune=False, persistent=persistent)
    assert all(r.layout().values())
    passes = dict(r.info())
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    big = int(np.nonzero(lengths == 1 << 14)[0][1])
    small = int(np.nonzero(lengths == 512)[0][0])
    r.set_fault(big, mode=t.TFFT_FAULT_SCALE, pass_=passes[1 << 14] - 1, stage=0, line=2, index=7, factor=2.0)
    r.set_fault(small, mode=t.TFFT_FAULT_SCALE, pass_=0, stage=1, line=0, index=11, factor=2.0)
    r.exec(xt, yt)
    torch.cuda.synchronize()
    _check(lengths, x, yt.cpu().numpy(), xg, yg)
    st = r.report()
    assert st["detected"] == 2 and st["corrected"] + st["recomputed"] == 2, st
    r.destroy()


def test_ragged_complex128_in_place():
    """complex128 buckets addressed in place (offsets multiples of 64
    elements), N(0,1) re/im, a fault corrected, against the oracle at the
    complex128 tolerance."""
    import torch
    rng = np.random.default_rng(1212)
    lengths = (1 << rng.integers(6, 14, size=120)).astype(np.int64)
    total = int(lengths.sum())
    x = rng.standard_normal(total) + 1j * rng.standard_normal(total)
    r = t.Ragged(lengths.tolist(), dtype=t.TFFT_C128, autotune=False)
    assert all(r.layout().values()), r.layout()
    passes = dict(r.info())
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    yg = Guarded(x.shape, xg.t.dtype)
    xt, yt = xg.t, yg.t
    sig = int(np.nonzero(lengths == 4096)[0][1])
    r.set_fault(sig, mode=t.TFFT_FAULT_SCALE, pass_=passes[4096] - 1, stage=0, line=0, index=6, factor=1.25)
    r.exec(xt, yt)
    torch.cuda.synchronize()
    y = yt.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    for n in np.unique(lengths):
        idx = np.nonzero(lengths == n)[0]
        xs = np.stack([x[off[i]:off[i] + n] for i in idx])
        ys = np.stack([y[off[i]:off[i] + n] for i in idx])
        assert rel_err_rows(ys, oracle.fft(xs)).max() <= tol(int(n), t.TFFT_C128), int(n)
    xg.check("input"); yg.check("output")
    st = r.report()
    assert st["detected"] == 1 and st["corrected"] + st["recomputed"] == 1, st
    r.destroy()


def test_persistent_families_match_bucket_streams_bitwise():
    """The pass families run the same tile-kernel body on the same chunks as
    the buckets' own launches: the outputs agree bit for bit, clean, over
    two execs (the second a graph replay)."""
    import torch
    lengths, x = _ragged_input(1500, seed=31, lo=6, hi=16)
    xg = Guarded(x.shape, None, fill=torch.from_numpy(x).cuda())
    outs = []
    for persistent in (False, True):
        r = t.Ragged(lengths.tolist(), autotune=False, persistent=persistent)
        yg = Guarded(x.shape, xg.t.dtype)
        for _ in range(2):
            yg.t.zero_()
            r.exec(xg.t, yg.t)
            torch.cuda.synchronize()
            outs.append(yg.t.cpu().numpy())
        yg.check("ragged output")
        st = r.report()
        assert st["detected"] == 0, st
        r.destroy()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[2], outs[3])
    assert np.array_equal(outs[0], outs[2])
    _check(lengths, x, outs[2], xg)
