"""Host-side helpers of bench.py on CPU: the ragged fault sites (one per 1000
signals, distinct checksum groups, at most four per length and one below 256
points), the one-N-per-step cycle of the reference arm, the oracle process
pool, and the recorded DRAM traffic lookup."""
import json
import os

import numpy as np

import bench


def test_ragged_fault_sites_distinct_groups():
    rng = np.random.default_rng(5)
    lengths = (1 << rng.integers(6, 17, size=20000)).astype(np.int64)
    sites = bench.ragged_fault_sites(lengths, 1, seed=5)
    assert len(sites) == 20
    local, counts = {}, {}
    for i, n in enumerate(lengths):
        local[i] = counts.get(int(n), 0)
        counts[int(n)] = local[i] + 1
    groups = {(int(lengths[i]), local[i] // 16) for i in sites}
    assert len(groups) == len(sites)                  # one fault per checksum group
    per_len = {}
    for i in sites:
        per_len[int(lengths[i])] = per_len.get(int(lengths[i]), 0) + 1
    assert all(c <= (1 if n < 256 else 4) for n, c in per_len.items())


def test_oracle_pool_runs_one_sample_per_process():
    pool = bench.OraclePool(2)
    try:
        f, s, desc = pool.sample(1 << 10, sweep=[8, 10])
    finally:
        pool.close()
    # each process transforms 4 signals of 256 and 1 of 1024 points
    assert f == 2 * (bench.flops(256, 4) + bench.flops(1024, 1))
    assert s > 0 and "2 processes" in desc


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    rec = {"kernel_source_hash": bench.kernel_source_hash(), "bytes_per_launch": {"first_pass": 1230},
           "bench_elements_per_launch": 1 << 28}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["kernel_source_hash"])
    assert bench.recorded_traffic("first_pass", 1 << 28) == 1230
    assert bench.recorded_traffic("first_pass", 1 << 27) == 615     # bytes scale with the launch
    assert bench.recorded_traffic("single_pass", 1 << 28) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.recorded_traffic("first_pass", 1 << 28) is None


def test_host_cores_positive():
    assert bench.host_cores() >= 1
    assert bench.host_cores() <= (os.cpu_count() or 1)


def test_min_passes_follows_the_tile_and_two_pass_limits():
    # one 4096-point tile, two passes of at most 8192-point sub-transforms
    # (2^26 = 8192^2), three beyond
    assert [bench.min_passes(1 << m) for m in (1, 8, 12)] == [1, 1, 1]
    assert [bench.min_passes(1 << m) for m in (13, 20, 24, 26)] == [2, 2, 2, 2]
    assert [bench.min_passes(1 << m) for m in (27, 29)] == [3, 3]


def test_c128_dft_flop_table_follows_the_radix2_recursion():
    # Dft<R> is two Dft<R/2> and R/2 butterflies: a complex add and subtract
    # (4 flops) after a multiply by omega_R^k, free for k = 0 and R/4, 4 flops
    # for the eighth roots (an add, a subtract, two multiplies by sqrt(1/2)),
    # 6 for the others (two multiplies and two multiply-adds)
    def root_flops(r, k):
        m = (k * (16 // r)) % 16
        if m % 4 == 0:
            return 0
        return 4 if m % 2 == 0 else 6

    def dft(r):
        if r == 1:
            return 0
        return 2 * dft(r // 2) + sum(4 + root_flops(r, k) for k in range(r // 2))

    assert {r: dft(r) for r in (1, 2, 4, 8, 16)} == bench.C128_DFT_FLOPS
    # a 4096-point single pass: radix-16 stages 16 x 16 x 16; two 64-point
    # passes: 8 x 8 each, plus the inter-pass twiddle and its recurrence
    one = bench.c128_executed_flops(4096, 1, {"passes": 1, "nsub": [4096], "stages": [3]})
    two = bench.c128_executed_flops(4096, 1, {"passes": 2, "nsub": [64, 64], "stages": [2, 2]})
    assert one == 4096 * (176 / 16 + 2 * (176 / 16 + 6 * 15 / 16))
    assert two == 4096 * (2 * (56 / 8 + 56 / 8 + 6 * 7 / 8) + 6 * (1 + 7 / 8))
