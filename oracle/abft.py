"""Two-sided ABFT of TurboFFT (Section III), restated step by step in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation (Section III-A, Eq. two_side_X / two_side_Y): the batch is the matrix
X = [x_0 ... x_{B-1}] (one signal per column), Y = W X with W the DFT matrix.
Signals are split into checksum groups of G consecutive signals; inside a
group b = 0..G-1.

* Signal-side (left) encoding vector r: Wang's e_Wang, r_j = w3^j with
  w3 = e^{-2 pi i/3} (Section II, "ABFT scheme"), or a seeded random +-1
  vector (the sign of bit 63 of output j of a SplitMix64 stream, Steele, Lea
  and Flood, OOPSLA 2014), or their product s_j w3^j ("signed e_Wang").  Its image through the DFT is the checksum vector
  w = W^T r = W r (W is symmetric).
* Batch-side (right) encoding vectors: e_1 = ones and the index weights
  e_3 = (1, 2, ..., G) (Section III, "another encoding vector e_3").
* Input checksums   S1 = w^T (X e_1),  S2 = w^T (X e_3).
* Output checksums  T1 = r^T (Y e_1),  T2 = r^T (Y e_3).
* Detect: |T1 - S1| > tau (Section II "checksum test with threshold delta").
* Locate: with a single faulty column b*, T2 - S2 = (b*+1)(T1 - S1), so
  b* = round(Re q) - 1 with q = (T2 - S2)/(T1 - S1) ("the corrupted input can
  be located using a quotient").
* Correct (Section III-B, delayed batched correction): the divergence of the
  batch checksum, delta = Y' e_1 - W (X e_1), is subtracted from column b*.

Readings of points the paper leaves open:
  - tau = kappa * u * (log2(N) + 4) * sqrt(N) * sqrt(sum_b ||x_b||^2): an
    absolute, Parseval-scaled threshold (the +4 covers the rounding of the
    checksum arithmetic itself); the paper prints no value for delta.
  - The correction is evaluated as y_{b*} = W(X e_1) - sum_{b != b*} y'_b,
    which equals y'_{b*} - delta exactly in real arithmetic and stays exact
    when the fault is huge or non-finite.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fft as _fft

W3 = complex(-0.5, -0.86602540378443864676372317075293618)   # e^{-2 pi i/3}


def left_vector(n: int) -> np.ndarray:
    """r_j = w3^j, j = 0..N-1 (e_Wang).  Only j mod 3 matters."""
    j = np.arange(n) % 3
    table = np.array([1.0 + 0j, W3, W3.conjugate()])   # w3^0, w3^1, w3^2
    return table[j]


_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 generator whose state
    starts at `seed`: output k = mix(seed + (k+1) gamma) with the published
    constants (gamma = 0x9E3779B97F4A7C15, multipliers 0xBF58476D1CE4E5B9 and
    0x94D049BB133111EB, shifts 30, 27, 31), all arithmetic modulo 2^64."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def random_left_vector(n: int, seed: int) -> np.ndarray:
    """r_k = +1 when bit 63 of SplitMix64 output k is 0, else -1."""
    bits = splitmix64(seed, n) >> np.uint64(63)
    return np.where(bits == 0, 1.0, -1.0).astype(np.complex128)


def vectors(n: int, kind: str = "wang", seed: int = 0):
    """(r, w) for kind 'wang' (e_Wang, w in closed form), 'random' (+-1
    signs) or 'signed_wang' (r_k = s_k w3^k, the random signs times e_Wang);
    for the random kinds w = W r with the oracle FFT."""
    if kind == "wang":
        return left_vector(n), checksum_vector_closed_form(n)
    if kind == "random":
        r = random_left_vector(n, seed)
        return r, _fft(r)
    if kind == "signed_wang":
        r = random_left_vector(n, seed) * left_vector(n)
        return r, _fft(r)
    raise ValueError(kind)


def checksum_vector_closed_form(n: int) -> np.ndarray:
    """w_k = sum_j w3^j wN^{jk} = (1 - w3^N) / (1 - w3 wN^k): a finite
    geometric series (wN = e^{-2 pi i/N}); no term vanishes since 3 does not
    divide N = 2^m.

    The denominator is evaluated without cancellation near its zero
    (k ~ 2N/3): w3 wN^k = e^{-i theta} with theta = 2 pi m / (3N),
    m = (N + 3k) mod 3N an exact integer, and 1 - e^{-i theta} =
    2 sin(theta/2) (sin(theta/2) + i cos(theta/2)); theta/2 is folded to
    [0, pi/2] first (sin(pi - a) = sin a, cos(pi - a) = -cos a) so that sin is
    never taken of an argument near pi."""
    k = np.arange(n, dtype=np.int64)
    m = (n + 3 * k) % (3 * n)
    upper = 2 * m > 3 * n
    mm = np.where(upper, 3 * n - m, m)
    half = np.pi * mm.astype(np.float64) / (3.0 * n)
    s = np.sin(half)
    c = np.where(upper, -np.cos(half), np.cos(half))
    denom = 2.0 * s * (s + 1j * c)
    w3_n = left_vector(n + 1)[n]          # w3^N through the mod-3 table
    return (1.0 - w3_n) / denom


def checksum_vector_by_fft(n: int) -> np.ndarray:
    """w = W r computed with the oracle FFT (W symmetric, so W^T r = W r)."""
    return _fft(left_vector(n))


def index_weights(g: int) -> np.ndarray:
    """e_3 = (1, 2, ..., G) across the group (Section III)."""
    return np.arange(1, g + 1, dtype=np.float64)


@dataclass
class GroupChecksums:
    S1: complex
    S2: complex
    T1: complex
    T2: complex
    energy: float          # sum_b ||x_b||^2 of the group


def group_checksums(xg: np.ndarray, yg: np.ndarray, w: np.ndarray | None = None,
                    r: np.ndarray | None = None) -> GroupChecksums:
    """Encode one group: xg, yg are (G, N) inputs and (possibly faulty)
    outputs.  Right side first (X e_1, X e_3), then the left dot products."""
    xg = np.asarray(xg, dtype=np.complex128)
    yg = np.asarray(yg, dtype=np.complex128)
    g, n = xg.shape
    if w is None:
        w = checksum_vector_closed_form(n)
    if r is None:
        r = left_vector(n)
    e1 = np.ones(g)
    e3 = index_weights(g)
    with np.errstate(over="ignore", invalid="ignore"):
        return _group_checksums(xg, yg, w, r, e1, e3)


def _group_checksums(xg, yg, w, r, e1, e3):
    c1 = e1 @ xg                       # X e_1, length N
    c2 = e3 @ xg                       # X e_3
    d1 = e1 @ yg                       # Y e_1
    d2 = e3 @ yg                       # Y e_3
    return GroupChecksums(S1=complex(w @ c1), S2=complex(w @ c2),
                          T1=complex(r @ d1), T2=complex(r @ d2),
                          energy=float(np.sum(np.abs(xg) ** 2)))


def threshold(n: int, energy: float, u: float, kappa: float) -> float:
    """tau = kappa * u * (log2(N) + 4) * sqrt(N) * sqrt(energy)."""
    log2n = int(round(np.log2(n)))
    return kappa * u * (log2n + 4) * np.sqrt(n) * np.sqrt(energy)


@dataclass
class GroupVerdict:
    detected: bool
    located: int           # b* in 0..G-1, or -1 when not locatable
    residual: float        # |T1 - S1|
    tau: float
    quotient: complex


def verify_group(cs: GroupChecksums, n: int, g: int, u: float, kappa: float) -> GroupVerdict:
    """Detect then locate (quotient) for one group."""
    d1 = cs.T1 - cs.S1
    d2 = cs.T2 - cs.S2
    tau = threshold(n, cs.energy, u, kappa)
    res = abs(d1)
    finite = np.isfinite(d1) and np.isfinite(d2)
    detected = (not finite) or res > tau
    q = complex("nan+nanj")
    located = -1
    if detected and finite and d1 != 0:
        q = d2 / d1
        m = int(np.rint(q.real))
        if abs(q.real - m) < 0.25 and abs(q.imag) < 0.25 and 1 <= m <= g:
            located = m - 1
    return GroupVerdict(detected=bool(detected), located=located, residual=float(res),
                        tau=float(tau), quotient=q)


def signal_residuals(xg: np.ndarray, yg: np.ndarray, w: np.ndarray, r: np.ndarray):
    """Left-side residual of every signal of a group, d_b = r^T y'_b - w^T x_b
    (the one-sided check of Section III applied to each column), and its
    input energy E_b = ||x_b||^2.  The group's two-sided residuals are their
    right-side encodings: T1 - S1 = sum_b d_b (e_1) and T2 - S2 = sum_b (b+1)
    d_b (e_3)."""
    xg = np.asarray(xg, dtype=np.complex128)
    yg = np.asarray(yg, dtype=np.complex128)
    with np.errstate(over="ignore", invalid="ignore"):
        d = yg @ r - xg @ w
    return d, np.sum(np.abs(xg) ** 2, axis=1)


@dataclass
class SignalVerdict:
    detected: bool
    located: int           # b* in 0..G-1, or -1 (recompute the group)
    flagged: list          # signals whose own test failed
    group_residual: float  # |sum_b d_b| = |T1 - S1|
    group_tau: float
    quotient: complex      # sum_b (b+1) d_b / sum_b d_b


def verify_group_signals(xg: np.ndarray, yg: np.ndarray, w: np.ndarray, r: np.ndarray, n: int,
                         u: float, kappa: float) -> SignalVerdict:
    """Detection and location from per-signal residuals.

    Each signal b is tested on its own, |d_b| > tau(E_b) with the threshold of
    :func:`threshold` taken over that signal's energy (or d_b not finite); the
    group is also tested with its two-sided residual |sum_b d_b| > tau(sum_b
    E_b).  Location: the one signal whose own test failed; with none failing
    (a detection by the group test alone) the quotient of Section III,
    sum_b (b+1) d_b / sum_b d_b = b* + 1; with several failing, none (the
    group is recomputed: more than one fault)."""
    d, e = signal_residuals(xg, yg, w, r)
    g = d.shape[0]
    tau_b = threshold(n, 1.0, u, kappa) * np.sqrt(e)
    finite = np.isfinite(d)
    with np.errstate(invalid="ignore"):
        flagged = [b for b in range(g) if (not finite[b]) or abs(d[b]) > tau_b[b]]
    dfin = np.where(finite, d, 0.0)
    D1 = complex(np.sum(dfin))
    D2 = complex(np.sum(np.arange(1, g + 1) * dfin))
    tau_g = threshold(n, float(np.sum(np.where(finite, e, 0.0))), u, kappa)
    res = abs(D1)
    detected = bool(flagged) or res > tau_g
    q = D2 / D1 if D1 != 0 else complex("nan+nanj")
    located = -1
    if detected:
        if len(flagged) == 1:
            located = flagged[0]
        elif not flagged and D1 != 0:
            m = int(np.rint(q.real))
            if abs(q.real - m) < 0.25 and abs(q.imag) < 0.25 and 1 <= m <= g:
                located = m - 1
    return SignalVerdict(detected=detected, located=located, flagged=flagged, group_residual=float(res),
                         group_tau=float(tau_g), quotient=q)


def second_left_vector(n: int, kind: str = "signed_wang", seed: int = 0, radix: int = 16) -> np.ndarray:
    """r2_k = r_k w3^floor(radix k / N): the left vector of :func:`vectors`
    times a phase that steps with the top bits of k (radix = the radix of the
    transform's last stage, 16 for complex64 and 8 for complex128 here)."""
    r, _ = vectors(n, kind, seed)
    k = np.arange(n, dtype=np.int64)
    return r * left_vector(radix)[(radix * k) // n]


def last_pass_vector(n: int, n_last: int, seed: int, kind: str = "signed_wang", radix: int = 16) -> tuple:
    """(r2, u2) of the second check across the last pass of a multi-pass
    transform.  The last pass takes the line of output class L (outputs
    L + M k, M = N / n_last) from its input z[L] by an n_last-point DFT, so
    r2^T y = sum_L u2[L] . z[L] with u2[L][m] = sum_k r2[L + M k] w^(m k)
    (w = e^{-2 pi i / n_last}); r2 is :func:`second_left_vector`."""
    r2 = second_left_vector(n, kind, seed, radix)
    m_cls = n // n_last
    rows = r2.reshape(n_last, m_cls).T            # rows[L][k] = r2[L + M k]
    return r2, _fft(rows)


def locate_nonfinite(xg: np.ndarray, yg: np.ndarray, r=None, w=None) -> int:
    """When the group residual is not finite (a value or a checksum sum
    overflowed) the quotient is undefined.  The faulty column is then the
    unique signal holding a non-finite value or, if every value is finite,
    the signal whose own left residual |r^T y'_b - w^T x_b| is largest,
    evaluated on data scaled by its largest magnitude so the sums cannot
    overflow.  Returns -1 if several signals hold non-finite values."""
    xg = np.asarray(xg, dtype=np.complex128)
    yg = np.asarray(yg, dtype=np.complex128)
    bad = [b for b in range(yg.shape[0]) if not np.all(np.isfinite(yg[b]))]
    if len(bad) == 1:
        return bad[0]
    if bad:
        return -1
    n = yg.shape[1]
    scale = max(1.0, float(np.max(np.abs(yg))), float(np.max(np.abs(xg))))
    if r is None:
        r, w = left_vector(n), checksum_vector_closed_form(n)
    res = [abs(r @ (yg[b] / scale) - w @ (xg[b] / scale)) for b in range(yg.shape[0])]
    return int(np.argmax(res))


def correct_group(xg: np.ndarray, yg: np.ndarray, bstar: int) -> np.ndarray:
    """Section III-B correction of column b*: y_{b*} = W(X e_1) - sum_{b!=b*} y'_b
    (= y'_{b*} - (Y' e_1 - W X e_1)).  Returns a corrected copy of yg."""
    xg = np.asarray(xg, dtype=np.complex128)
    yc = np.array(yg, dtype=np.complex128, copy=True)
    g = xg.shape[0]
    f_c1 = _fft(np.ones(g) @ xg)                      # W (X e_1)
    others = [b for b in range(g) if b != bstar]
    yc[bstar] = f_c1 - (np.sum(yc[others], axis=0) if others else 0.0)
    return yc


@dataclass
class BatchResult:
    y: np.ndarray                  # corrected outputs
    detected_groups: list
    located: dict                  # group -> b* (global signal index)
    uncorrectable_groups: list


def run(x: np.ndarray, y_faulty: np.ndarray, group: int, u: float, kappa: float,
        kind: str = "wang", seed: int = 0, per_signal: bool = False) -> BatchResult:
    """Apply the whole scheme to a batch: groups of ``group`` consecutive
    signals (the last one may be shorter), detect, locate, correct, with the
    signal-side vector of ``kind`` (see :func:`vectors`); ``per_signal``
    detects and locates with :func:`verify_group_signals` instead of the
    group checksums alone."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.array(y_faulty, dtype=np.complex128, copy=True)
    bsz, n = x.shape
    r, w = vectors(n, kind, seed)
    det, loc, unc = [], {}, []
    for g0 in range(0, bsz, group):
        g1 = min(bsz, g0 + group)
        gi = g0 // group
        if per_signal:
            sv = verify_group_signals(x[g0:g1], y[g0:g1], w, r, n, u, kappa)
            if not sv.detected:
                continue
            det.append(gi)
            if sv.located < 0:
                unc.append(gi)
                continue
            loc[gi] = g0 + sv.located
            y[g0:g1] = correct_group(x[g0:g1], y[g0:g1], sv.located)
            continue
        cs = group_checksums(x[g0:g1], y[g0:g1], w=w, r=r)
        v = verify_group(cs, n, g1 - g0, u, kappa)
        if not v.detected:
            continue
        det.append(gi)
        b = v.located
        if b < 0 and not (np.isfinite(cs.T1) and np.isfinite(cs.T2)):
            b = locate_nonfinite(x[g0:g1], y[g0:g1], r, w)
        if b < 0:
            unc.append(gi)
            continue
        loc[gi] = g0 + b
        y[g0:g1] = correct_group(x[g0:g1], y[g0:g1], b)
    return BatchResult(y=y, detected_groups=det, located=loc, uncorrectable_groups=unc)
