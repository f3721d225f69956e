"""The autotuner and the tile-threads option on the GPU.  The 256- and
512-thread tile kernels run the same butterflies on the same lines (only
the lines a tile differ), so their outputs agree bit for bit and both meet
the oracle's tolerance; the autotuner's choice is at least as fast as the
planner's own (it is one of the candidates), and a later plan of the same
transform is built with it and stays correct."""
import numpy as np
import pytest

import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("log2n,batch,first", [(17, 4, 8), (17, 4, 9), (18, 2, 9), (20, 2, 11), (20, 2, 9),
                                               (19, 2, 10)])
def test_256_and_512_thread_tiles_agree_bitwise_and_with_oracle(log2n, batch, first):
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=log2n + first).astype(np.complex64)
    ref = oracle_fft(x)
    ys, infos = [], []
    for threads in (256, 512):
        y, p = run_gpu(x, t.TFFT_C64, first_pass_log2=first, tile_threads=threads)
        try:
            infos.append(t.tfft_plan_info(p))
            assert t.tfft_report(p) == (0, 0)
        finally:
            t.tfft_destroy(p)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
        ys.append(y)
    # each takes its own form where it has a kernel for the pass, else the other
    wide = [512 <= s <= 2048 for s in infos[1]["nsub"][:2]]
    assert all(th in (256, 512) for info in infos for th in info["tile_threads"][:2])
    assert all(th == 512 for th, w in zip(infos[1]["tile_threads"], wide) if w)
    assert infos[0]["tile_threads"][:2] != infos[1]["tile_threads"][:2]
    assert np.array_equal(ys[0], ys[1])


def test_512_thread_tiles_detect_and_correct_a_fault():
    n, batch = 1 << 20, 2
    x = uniform_batch(n, batch, seed=5).astype(np.complex64)
    fault = dict(mode=t.TFFT_FAULT_BITFLIP, pass_=1, stage=1, signal=1, line=77, index=300, bit=28)
    y, p = run_gpu(x, t.TFFT_C64, tile_threads=512, fault=fault)
    try:
        assert t.tfft_plan_info(p)["tile_threads"][:2] == [512, 512]
        assert t.tfft_report(p) == (1, 1)
    finally:
        t.tfft_destroy(p)
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)


def test_autotune_choice_is_recorded_reused_and_correct(tmp_path, monkeypatch):
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TFFT_TUNE_CACHE", str(cache))
    t.tfft_tune_clear()
    try:
        n, batch = 1 << 17, 64
        x = uniform_batch(n, batch, seed=11).astype(np.complex64)
        xt = torch.from_numpy(x).cuda()
        yt = torch.empty_like(xt)
        r = t.tfft_autotune(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, xt, yt, reps=3)
        assert r["candidates"] >= 4
        assert 0 < r["ms"] <= r["default_ms"]
        assert r["passes"] in (2, 3) and r["tile_threads"] in (256, 512)
        assert (r["first_pass_log2"] > 0) == (r["passes"] == 2)
        assert t.tfft_tune_lookup(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED) == (
            r["passes"], r["first_pass_log2"], r["tile_threads"])
        fields = cache.read_text().split()
        assert fields[0] == "tfft-tune-1" and [int(v) for v in fields[1:9]] == [
            n, batch, 0, 2, 0, r["passes"], r["first_pass_log2"], r["tile_threads"]]
        # a plan that leaves the configuration to the planner now takes it
        y, p = run_gpu(x, t.TFFT_C64)
        try:
            info = t.tfft_plan_info(p)
            assert info["tuned"] == 1 and info["passes"] == r["passes"]
            if r["passes"] == 2:
                assert info["nsub"][0] == 1 << r["first_pass_log2"]
            assert t.tfft_report(p) == (0, 0)
        finally:
            t.tfft_destroy(p)
        assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
        # ... and one that forces any part of it does not
        y2, p2 = run_gpu(x, t.TFFT_C64, tile_threads=256)
        try:
            assert t.tfft_plan_info(p2)["tuned"] == 0
        finally:
            t.tfft_destroy(p2)
    finally:
        monkeypatch.delenv("TFFT_TUNE_CACHE")
        t.tfft_tune_clear()
    y3, p3 = run_gpu(x, t.TFFT_C64)
    try:
        assert t.tfft_plan_info(p3)["tuned"] == 0
    finally:
        t.tfft_destroy(p3)
