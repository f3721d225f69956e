"""Pins of the FP64 oracle against things other than itself.

Each test names what fixes the expected value: the DFT definition summed by
brute force, numpy's independent FFT, closed forms, textbook invariants, or
hand-worked fixtures in tests/golden/.  The oracle is only trusted because
these pass.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import abft

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)


def crandn(*shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def read_golden(name):
    blocks, cur = [], {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "N":
            cur = {"N": int(vals[0])}
            blocks.append(cur)
        else:
            v = np.array([float(t) for t in vals])
            cur[key] = v[0::2] + 1j * v[1::2]
    return blocks


# ---------------------------------------------------------------- FFT pins
@pytest.mark.parametrize("n", [1 << k for k in range(0, 9)])
def test_fft_matches_bruteforce_definition(n):
    """Section II definition summed directly in long double, N = 1..256."""
    x = crandn(3, n)
    assert rel(oracle.fft(x), oracle.dft_naive(x)) < 1e-15 * max(1, np.log2(n)) + 1e-16


@pytest.mark.parametrize("n", [1 << k for k in range(1, 9)])
def test_inverse_matches_bruteforce_definition(n):
    y = crandn(2, n)
    assert rel(oracle.ifft(y), oracle.dft_naive(y, sign=+1)) < 1e-15 * np.log2(n) + 1e-16


@pytest.mark.parametrize("n", [1 << k for k in (4, 10, 13, 16)])
def test_fft_matches_numpy_library(n):
    """numpy's pocketfft is an independent FFT implementation."""
    x = crandn(2, n)
    assert rel(oracle.fft(x), np.fft.fft(x, axis=-1)) < 1e-15 * np.log2(n)


def test_golden_hand_worked_dfts():
    for blk in read_golden("dft_small.txt"):
        y = oracle.fft(blk["x"])
        assert np.allclose(y, blk["y"], rtol=0, atol=1e-14), blk["N"]


@pytest.mark.parametrize("n", [2, 16, 1024, 1 << 15])
def test_delta_maps_to_constant_and_shifted_delta_to_column(n):
    x = np.zeros(n, complex); x[0] = 1.0
    assert np.max(np.abs(oracle.fft(x) - 1.0)) < 1e-15
    k = n // 2 + 1 if n > 2 else 1
    x = np.zeros(n, complex); x[k] = 1.0
    col = np.exp(-2j * np.pi * ((np.arange(n) * k) % n) / n)     # column k of W
    assert np.max(np.abs(oracle.fft(x) - col)) < 1e-14


@pytest.mark.parametrize("n,k0", [(64, 5), (4096, 1234), (1 << 16, 40000)])
def test_pure_tone_maps_to_one_bin(n, k0):
    t = np.arange(n)
    x = np.exp(2j * np.pi * ((k0 * t) % n) / n)
    y = oracle.fft(x)
    expect = np.zeros(n, complex); expect[k0] = n
    assert np.max(np.abs(y - expect)) < 1e-11 * n


@pytest.mark.parametrize("n", [8, 4096, 1 << 18])
def test_parseval_and_roundtrip(n):
    x = crandn(2, n)
    y = oracle.fft(x)
    assert abs(np.sum(np.abs(y) ** 2) / (n * np.sum(np.abs(x) ** 2)) - 1) < 1e-13
    assert rel(oracle.ifft(y), x) < 1e-15 * np.log2(n)


def test_linearity():
    n = 2048
    a, b = crandn(n), crandn(n)
    alpha, beta = 0.3 - 1.7j, -2.5 + 0.25j
    lhs = oracle.fft(alpha * a + beta * b)
    rhs = alpha * oracle.fft(a) + beta * oracle.fft(b)
    assert rel(lhs, rhs) < 1e-14


def test_sizes_one_and_two_closed_form():
    a, b = 0.25 - 3j, 1.5 + 2j
    assert np.allclose(oracle.fft(np.array([a])), [a], atol=0)
    assert np.allclose(oracle.fft(np.array([a, b])), [a + b, a - b], atol=1e-15)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, complex))


# ---------------------------------------------------------- checksum pins
@pytest.mark.parametrize("n", [4, 256, 1024, 1 << 14])
def test_checksum_vector_two_independent_ways(n):
    """Closed-form geometric sum vs the DFT of r (absolute error of the FFT
    route is ~u sqrt(N) log2 N; the closed form is accurate to a few u)."""
    a = abft.checksum_vector_closed_form(n)
    b = abft.checksum_vector_by_fft(n)
    eps = np.finfo(np.float64).eps
    assert np.all(np.abs(a - b) <= 4 * eps * (np.abs(b) + np.sqrt(n) * np.log2(n)))
    assert np.min(np.abs(a)) > 0.86        # never zero for N = 2^m


def test_checksum_vector_golden_n4():
    blk = read_golden("checksum_small.txt")[0]
    assert np.allclose(abft.checksum_vector_closed_form(4), blk["w"], atol=1e-14)
    assert np.allclose(abft.checksum_vector_by_fft(4), blk["w"], atol=1e-14)


@pytest.mark.parametrize("n", [16, 1024, 1 << 16])
def test_left_checksum_identity(n):
    """(r^T W) x = r^T (W x) for any x (Eq. ABFT / C)."""
    x = crandn(n)
    w = abft.checksum_vector_closed_form(n)
    lhs = w @ x
    rhs = abft.left_vector(n) @ oracle.fft(x)
    assert abs(lhs - rhs) / (np.sqrt(n) * np.linalg.norm(x)) < 1e-14


def test_all_ones_left_vector_sums_to_n_x0():
    """Textbook special case: sum_k y_k = N x_0 (why e = ones is weak)."""
    n = 512
    x = crandn(n)
    assert abs(np.sum(oracle.fft(x)) - n * x[0]) < 1e-11 * n


# ------------------------------------------------------------ ABFT pins
def _clean_group(n, g, seed):
    r = np.random.default_rng(seed)
    x = r.uniform(-1, 1, (g, n)) + 1j * r.uniform(-1, 1, (g, n))
    return x, oracle.fft(x)


def test_clean_group_is_not_detected():
    for seed in range(20):
        x, y = _clean_group(256, 8, seed)
        cs = abft.group_checksums(x, y)
        v = abft.verify_group(cs, 256, 8, u=2.0 ** -53, kappa=4.0)
        assert not v.detected


@pytest.mark.parametrize("n,g", [(8, 1), (16, 4), (64, 8)])
def test_every_site_detected_located_corrected(n, g):
    """Brute force over every (signal, element) output site: an exact fault
    gives the quotient b*+1, and the correction recovers W x."""
    x, y = _clean_group(n, g, 7)
    for b in range(g):
        for j in range(n):
            yf = y.copy()
            yf[b, j] += 0.3 - 0.2j
            cs = abft.group_checksums(x, yf)
            v = abft.verify_group(cs, n, g, u=2.0 ** -53, kappa=4.0)
            assert v.detected and v.located == b, (b, j, v)
            assert abs(v.quotient - (b + 1)) < 1e-9
            yc = abft.correct_group(x, yf, b)
            assert rel(yc, y) < 1e-14


def test_weight_zero_would_hide_signal_zero():
    """Plant the e_3 indexing mistake (weights 0..G-1) in a copy: the quotient
    for a fault in signal 0 becomes 0 and cannot name it -- the reason the
    weights are 1..G."""
    n, g = 32, 4
    x, y = _clean_group(n, g, 3)
    yf = y.copy(); yf[0, 5] += 1.0
    d1 = abft.left_vector(n) @ (np.ones(g) @ (yf - y))
    d2 = abft.left_vector(n) @ (np.arange(g) @ (yf - y))
    assert abs(d2 / d1) < 1e-12
    cs = abft.group_checksums(x, yf)
    assert abft.verify_group(cs, n, g, 2.0 ** -53, 4.0).located == 0


def test_planted_sign_error_in_w_is_caught():
    """Plant a conjugated e_Wang (w3^{+j}) in the left vector: the identity
    pin fails, so a wrong sign cannot slip through."""
    n = 64
    x = crandn(n)
    bad_r = np.conj(abft.left_vector(n))
    lhs = abft.checksum_vector_closed_form(n) @ x
    assert abs(lhs - bad_r @ oracle.fft(x)) > 1e-3


@pytest.mark.parametrize("stage", [-1, 0, 3, 5])
@pytest.mark.parametrize("bit", [20, 45, 62])
def test_emulated_bitflip_fp64_detected_and_corrected(stage, bit):
    """Section II-A fault model run on the CPU: one bit flipped in an
    intermediate FP64 value of signal 2; large flips are caught and fixed."""
    n, g, bs = 64, 4, 2
    x, y = _clean_group(n, g, 11)
    yf = y.copy()
    yf[bs] = oracle.fft_faulty(x[bs], 64, stage=stage, elem=13, comp=1, bit=bit)
    err = np.linalg.norm(yf[bs] - y[bs]) / np.linalg.norm(y[bs])
    with np.errstate(all='ignore'):
        res = abft.run(x, yf, group=g, u=2.0 ** -53, kappa=4.0)
    if not np.isfinite(err) or err > 1e-12:
        assert res.detected_groups == [0]
        assert res.located == {0: bs}
        assert rel(res.y, y) < 1e-12
    else:
        assert rel(res.y, y) < 1e-12     # benign: output already within tolerance


def test_fp32_emulation_clean_matches_within_fp32_rounding():
    n = 1024
    x, y = _clean_group(n, 1, 5)
    y32 = oracle.fft_faulty(x[0].astype(np.complex64), 32)
    assert 1e-9 < rel(y32, y[0]) < 2e-6 * np.log2(n)


def test_nonfinite_fault_located_by_scan():
    n, g = 32, 4
    x, y = _clean_group(n, g, 9)
    yf = y.copy(); yf[3, 7] = np.inf
    res = abft.run(x, yf, group=g, u=2.0 ** -53, kappa=4.0)
    assert res.detected_groups == [0] and res.located == {0: 3}
    assert rel(res.y, y) < 1e-13


def test_ragged_last_group():
    n, B, g = 16, 11, 4
    r = np.random.default_rng(1)
    x = r.standard_normal((B, n)) + 1j * r.standard_normal((B, n))
    y = oracle.fft(x)
    yf = y.copy(); yf[10, 2] *= 1.01
    res = abft.run(x, yf, group=g, u=2.0 ** -53, kappa=4.0)
    assert res.detected_groups == [2] and res.located == {2: 10}
    assert rel(res.y, y) < 1e-13


# ------------------------------------------------ random signal-side vector
def test_splitmix64_golden_outputs():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    expect = [int(v, 16) for v in lines[1][1:]]
    got = [int(v) for v in abft.splitmix64(seed, 3)]
    assert got == expect


def test_splitmix64_counter_matches_sequential_stream():
    """output k started at `start` equals output start+k of the stream."""
    a = abft.splitmix64(12345, 10)
    b = abft.splitmix64(12345, 4, start=6)
    assert list(a[6:]) == list(b)


def test_random_vector_is_balanced_and_flat():
    """+-1 signs, about half each; W r has no systematically small entry
    (|w_k|^2 averages N by Parseval)."""
    n = 1 << 14
    r, w = abft.vectors(n, "random", seed=20240502)
    assert set(np.unique(r.real)) == {-1.0, 1.0} and np.all(r.imag == 0)
    assert abs(np.mean(r.real)) < 4 / np.sqrt(n)
    assert abs(np.mean(np.abs(w) ** 2) / n - 1) < 1e-12
    assert np.mean(np.abs(w) < 0.05 * np.sqrt(n)) < 0.01


@pytest.mark.parametrize("kind", ["wang", "random"])
def test_identity_holds_for_both_vectors(kind):
    n = 4096
    r, w = abft.vectors(n, kind, seed=7)
    x = crandn(n)
    assert abs(w @ x - r @ oracle.fft(x)) / (np.sqrt(n) * np.linalg.norm(x)) < 1e-14


def test_random_vector_detects_early_stage_fault_wang_misses():
    """A small input-stage fault at a position where |w_Wang| is minimal:
    e_Wang's residual stays below the threshold, the random vector's does not
    (the blind band of e_Wang)."""
    n, g = 1 << 12, 4
    x, y = _clean_group(n, g, 21)
    rw, ww = abft.vectors(n, "wang")
    k = int(np.argmin(np.abs(ww)))                      # |w_k| ~ 0.87
    eps = 2e-3
    xf = x.copy(); xf[1, k] += eps
    yf = y.copy(); yf[1] = oracle.fft(xf[1])             # fault before the FFT
    err = np.linalg.norm(yf[1] - y[1]) / np.linalg.norm(y[1])
    assert err > 2e-6 * 12                               # harmful at FP32 tolerance
    u = 2.0 ** -24                                      # judged at FP32 noise
    cw = abft.group_checksums(x, yf, w=ww, r=rw)
    assert not abft.verify_group(cw, n, g, u, 1.0).detected
    rr, wr = abft.vectors(n, "random", seed=20240502)
    if abs(wr[k]) > 0.3 * np.sqrt(n):
        cr = abft.group_checksums(x, yf, w=wr, r=rr)
        v = abft.verify_group(cr, n, g, u, 1.0)
        assert v.detected and v.located == 1


def test_dft_bins_matches_definition_and_fft():
    """The spot-check oracle for long transforms equals the long-double
    definition and the radix-2 oracle on short ones, in both directions."""
    rng = np.random.default_rng(77)
    for n in (1, 2, 8, 256, 4096):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        ks = sorted(set(rng.integers(0, n, size=min(n, 12)).tolist()) | {0, n - 1})
        for sign in ((-1, 1) if n <= 256 else ()):
            # the definition oracle scales its inverse by 1/N; dft_bins does not
            ref = oracle.dft_naive(x[None, :], sign)[0] * (n if sign > 0 else 1)
            got = oracle.dft_bins(x, ks, sign, chunk=97)
            scale = np.linalg.norm(ref) / np.sqrt(n)
            assert np.max(np.abs(got - ref[ks])) <= 1e-12 * max(scale, 1e-300) * max(1, np.log2(n))
        y = oracle.fft(x[None, :])[0]
        assert np.allclose(oracle.dft_bins(x, ks), y[ks], rtol=0, atol=1e-11 * np.linalg.norm(y))


def test_late_butterfly_fault_projection_is_rarely_small():
    """Reading 5 (marginal faults): a fault in the last radix-16 butterfly of a
    signal changes 16 outputs k0 + q N/16 by delta w16^(q m); the checksum sees
    it through sum_q r_k delta w16^(q m), a sum of 16 random phases for the
    signed e_Wang vector.  Its magnitude relative to the fault's norm
    (4 |delta|) is Rayleigh-like: below 0.14 a few percent of the time (the
    threshold-to-norm ratio of a fault 1.04x the tolerance at N = 2^18), so
    such a fault can hide under the rounding noise, while below 0.01 almost
    never."""
    n = 1 << 14
    r, _ = abft.vectors(n, "signed_wang", seed=20240502)
    rng = np.random.default_rng(7)
    q = np.arange(16)
    ratios = []
    for _ in range(4000):
        k0 = int(rng.integers(n // 16))
        m = int(rng.integers(16))
        pattern = np.exp(-2j * np.pi * q * m / 16)
        proj = abs(np.sum(r[k0 + q * (n // 16)] * pattern))
        ratios.append(proj / 4.0)
    ratios = np.array(ratios)
    assert 0.005 < np.mean(ratios < 0.14) < 0.05
    assert np.mean(ratios < 0.01) < 0.002
    assert 0.8 < np.mean(ratios ** 2) < 1.2          # unit mean square: no systematic cancellation


@pytest.mark.parametrize("n", [2, 4, 8, 256, 4096])
def test_threshold_sits_above_fp32_rounding_noise(n):
    """Reading 4 (threshold): with kappa = 2, the residual |T1 - S1| of clean
    groups whose outputs carry FP32 rounding (the oracle's own FP32 radix-2
    emulation, a different operation order from any GPU kernel) stays well
    below tau = kappa u (log2 N + 4) sqrt(N) sqrt(E), over 40 groups of 16
    U[-1,1) signals."""
    rng = np.random.default_rng(11)
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    ratios = []
    for _ in range(40):
        xg = (rng.uniform(-1, 1, (16, n)) + 1j * rng.uniform(-1, 1, (16, n))).astype(np.complex64)
        yg = np.stack([oracle.fft_faulty(xg[b], 32) for b in range(16)])
        cs = abft.group_checksums(xg.astype(np.complex128), yg, w=w, r=r)
        v = abft.verify_group(cs, n, 16, 2.0 ** -24, 2.0)
        assert not v.detected
        ratios.append(v.residual / v.tau)
    assert max(ratios) < 0.6
    assert np.median(ratios) > 1e-3        # the residual is rounding noise, not exactly zero


def _bitrev(i, bits):
    return int(format(i, f"0{bits}b")[::-1], 2) if bits else 0


def _flip64(v, bit):
    u = np.array([v], dtype=np.float64).view(np.uint64)
    u ^= np.uint64(1) << np.uint64(bit)
    return float(u.view(np.float64)[0])


@pytest.mark.parametrize("n,elem,comp,bit", [(16, 3, 0, 52), (256, 77, 1, 60), (1024, 1000, 0, 45)])
def test_fault_emulation_input_flip_is_the_fft_of_the_flipped_input(n, elem, comp, bit):
    """Stage -1 of the fault emulation flips working element `elem` after the
    bit-reversal permutation, i.e. input x[bitrev(elem)]: the faulty
    transform equals the oracle FFT of the input with that bit flipped."""
    rng = np.random.default_rng(n + elem)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    pos = _bitrev(elem, int(np.log2(n)))
    xf = x.copy()
    if comp == 0:
        xf[pos] = complex(_flip64(x[pos].real, bit), x[pos].imag)
    else:
        xf[pos] = complex(x[pos].real, _flip64(x[pos].imag, bit))
    got = oracle.fft_faulty(x, 64, stage=-1, elem=elem, comp=comp, bit=bit)
    want = oracle.fft(xf)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("n,stage,elem", [(64, 0, 37), (256, 2, 100), (1024, 5, 613), (1024, 9, 88)])
def test_fault_emulation_stage_flip_spreads_over_its_residue_class(n, stage, elem):
    """After stage s of the radix-2 decimation-in-time transform the working
    array holds, in block i of length L = 2^(s+1), the L-point DFT Z_i of the
    input subsequence x[c + t N/L] with c = bitrev_{log2(N/L)}(i); the output
    is y_k = sum_i wN^(c k) Z_i[k mod L].  So a change delta of element
    elem = i L + m0 changes exactly the outputs k = m0 (mod L), by
    delta wN^(c k): a flip placed after the wrong stage or at the wrong
    position would change another set of outputs or another phase."""
    rng = np.random.default_rng(7 * n + stage)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lg = int(np.log2(n))
    L = 1 << (stage + 1)
    i, m0 = divmod(elem, L)
    c = _bitrev(i, lg - stage - 1)
    clean = oracle.fft_faulty(x, 64)
    bad = oracle.fft_faulty(x, 64, stage=stage, elem=elem, comp=0, bit=61)
    diff = bad - clean
    k = np.arange(n)
    phase = np.exp(-2j * np.pi * ((c * k) % n) / n)
    delta = diff[m0] / phase[m0]
    assert abs(delta) > 1e-3                      # the flip changed the value
    expect = np.where(k % L == m0, delta * phase, 0.0)
    assert np.max(np.abs(diff - expect)) <= 1e-9 * abs(delta)


# ------------------------------------------------ per-signal residuals
def _group(n, g, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, (g, n)) + 1j * rng.uniform(-1, 1, (g, n))).astype(dtype)


@pytest.mark.parametrize("n,g", [(64, 16), (1024, 16), (4096, 7)])
def test_signal_residuals_encode_to_the_group_checksums(n, g):
    """The right-side encodings of the per-signal residuals are the group
    residuals computed the other way round (right side first, then the left
    dot products): sum_b d_b = T1 - S1 and sum_b (b+1) d_b = T2 - S2."""
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    xg = _group(n, g, n + g)
    yg = oracle.fft(xg)
    yg[g // 2, 3] += 0.25 - 0.5j                  # any output, faulty or not
    d, e = abft.signal_residuals(xg, yg, w, r)
    cs = abft.group_checksums(xg, yg, w=w, r=r)
    scale = np.abs(cs.T1) + np.abs(cs.S1) + 1.0
    assert abs(np.sum(d) - (cs.T1 - cs.S1)) <= 1e-12 * scale
    assert abs(np.sum(np.arange(1, g + 1) * d) - (cs.T2 - cs.S2)) <= 1e-12 * g * scale
    assert np.allclose(e, np.sum(np.abs(xg) ** 2, axis=1))


@pytest.mark.parametrize("n,g", [(8, 1), (16, 4), (64, 8)])
def test_per_signal_every_site_detected_located_corrected(n, g):
    """Brute force over every (signal, output element) site: an exact-arithmetic
    fault of size 1e-3 of the signal's norm is detected by its own signal's
    test, named, and the correction restores the clean output."""
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    xg = _group(n, g, 3 * n + g)
    yc = oracle.fft(xg)
    for b in range(g):
        for k in range(n):
            yf = yc.copy()
            yf[b, k] += 1e-3 * np.linalg.norm(yc[b])
            v = abft.verify_group_signals(xg, yf, w, r, n, 2.0 ** -52, 2.0)
            assert v.detected and v.flagged == [b] and v.located == b, (b, k)
            fixed = abft.correct_group(xg, yf, b)
            assert np.linalg.norm(fixed - yc) <= 1e-10 * np.linalg.norm(yc)


@pytest.mark.parametrize("n", [2, 4, 8, 256, 4096])
def test_per_signal_threshold_sits_above_fp32_rounding_noise(n):
    """Clean groups whose outputs carry FP32 rounding (the oracle's FP32
    radix-2 emulation): no signal and no group is flagged with kappa = 2 and
    the largest per-signal ratio |d_b| / tau_b stays well below one."""
    rng = np.random.default_rng(12)
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    worst = 0.0
    for _ in range(20):
        xg = (rng.uniform(-1, 1, (16, n)) + 1j * rng.uniform(-1, 1, (16, n))).astype(np.complex64)
        yg = np.stack([oracle.fft_faulty(xg[b], 32) for b in range(16)])
        x64 = xg.astype(np.complex128)
        v = abft.verify_group_signals(x64, yg, w, r, n, 2.0 ** -24, 2.0)
        assert not v.detected
        d, e = abft.signal_residuals(x64, yg, w, r)
        worst = max(worst, float(np.max(np.abs(d) / (abft.threshold(n, 1.0, 2.0 ** -24, 2.0) * np.sqrt(e)))))
    assert worst < 0.6


def test_per_signal_test_catches_a_spread_fault_the_group_test_misses():
    """A fault spread over two outputs of one signal with a small projection on
    r (|r^T e| = 0.1 |delta|) and 1.5 times the tolerance in size: the group
    residual stays below the group threshold (it carries the rounding of all
    sixteen signals), the faulty signal's own residual exceeds its threshold
    (four times lower), so the per-signal scheme names and corrects it."""
    n, g = 256, 16
    u, kappa = 2.0 ** -24, 2.0
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    rng = np.random.default_rng(5)
    xg = (rng.uniform(-1, 1, (g, n)) + 1j * rng.uniform(-1, 1, (g, n))).astype(np.complex64)
    x64 = xg.astype(np.complex128)
    yg = np.stack([oracle.fft_faulty(xg[b], 32) for b in range(g)])
    ref = oracle.fft(x64)
    b, k1, k2, eps = 9, 17, 140, 0.1
    tol = 2e-6 * np.log2(n)
    delta = 1.5 * tol * np.linalg.norm(ref[b]) / np.sqrt(2.0)
    e = np.zeros(n, dtype=np.complex128)
    e[k1] = delta
    e[k2] = -delta * (r[k1] / r[k2]) * (1.0 - eps)
    yf = yg.copy()
    yf[b] += e
    err = np.linalg.norm(yf[b] - ref[b]) / np.linalg.norm(ref[b])
    assert err > tol                                       # harmful
    assert abs(r @ e) < 0.11 * abs(delta)                  # small projection
    grp = abft.verify_group(abft.group_checksums(x64, yf, w=w, r=r), n, g, u, kappa)
    assert not grp.detected                                # the group test alone misses it
    v = abft.verify_group_signals(x64, yf, w, r, n, u, kappa)
    assert v.detected and v.flagged == [b] and v.located == b
    res = abft.run(x64, yf, group=g, u=u, kappa=kappa, kind="signed_wang", seed=20240502, per_signal=True)
    assert res.located == {0: b}
    assert np.linalg.norm(res.y[b] - ref[b]) / np.linalg.norm(ref[b]) <= tol


def test_per_signal_two_faulty_signals_are_not_located():
    """Two signals whose own tests fail (outside the single-event model): the
    group is detected but not located, so it is recomputed."""
    n, g = 64, 8
    r, w = abft.vectors(n, "signed_wang", seed=20240502)
    xg = _group(n, g, 77)
    yf = oracle.fft(xg)
    yf[2, 5] += 1.0
    yf[6, 40] -= 0.5j
    v = abft.verify_group_signals(xg, yf, w, r, n, 2.0 ** -52, 2.0)
    assert v.detected and v.flagged == [2, 6] and v.located == -1


@pytest.mark.parametrize("n,n_last", [(64, 8), (1024, 32), (4096, 1024)])
def test_last_pass_vector_is_the_image_of_r2_through_the_last_pass(n, n_last):
    """For any last-pass input z (one row per output class L) the last pass's
    output, written out by its definition y[L + M k] = sum_m z[L][m] w^(m k),
    satisfies r2^T y = sum_{L, m} u2[L][m] z[L][m]."""
    r2, u2 = abft.last_pass_vector(n, n_last, seed=20240503)
    m_cls = n // n_last
    rng = np.random.default_rng(n)
    z = rng.standard_normal((m_cls, n_last)) + 1j * rng.standard_normal((m_cls, n_last))
    k = np.arange(n_last)
    y = np.empty(n, dtype=np.complex128)
    for L in range(m_cls):
        y[L + m_cls * k] = oracle.dft_naive(z[L])
    assert abs(r2 @ y - np.sum(u2 * z)) <= 1e-9 * np.sqrt(n) * np.linalg.norm(z)


def test_second_vector_sees_a_butterfly_fault_independently():
    """On the sixteen outputs c + q N/16 of a last-stage butterfly, a fault of
    the butterfly's input m is the tone A w16^(q m).  Its projections on r and
    on r2 = r w3^floor(16 k / N) are the sums of the same random signs at two
    frequencies a third of a cycle apart: over all classes and tones both are
    small together about as often as independent projections would be, and
    never both below a tenth of the fault's norm.  (The complex128 kernels'
    last stage has radix 8: r2 = r w3^floor(8 k / N), the same argument.)"""
    n = 1 << 14
    r, _ = abft.vectors(n, "signed_wang", seed=20240502)
    r2 = abft.second_left_vector(n, "signed_wang", seed=20240502)
    q = np.arange(16)
    p1, p2 = [], []
    for c in range(0, n // 16, 7):
        k = c + q * (n // 16)
        for m in range(16):
            tone = np.exp(-2j * np.pi * q * m / 16)
            p1.append(abs(r[k] @ tone) / 4.0)          # |r^T a| / ||a||
            p2.append(abs(r2[k] @ tone) / 4.0)
    p1, p2 = np.array(p1), np.array(p2)
    small1, small2 = p1 < 0.3, p2 < 0.3
    joint = np.mean(small1 & small2)
    assert np.mean(small1) > 0.02 and np.mean(small2) > 0.02      # each alone has a tail
    assert joint <= 3.0 * np.mean(small1) * np.mean(small2) + 1e-3
    assert np.max(np.minimum(p1, p2)) > 0.5 and np.min(np.maximum(p1, p2)) > 0.1
    assert abs(np.corrcoef(p1, p2)[0, 1]) < 0.2
