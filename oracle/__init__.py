"""FP64 CPU oracle for the batched 1-D C2C FFT and its two-sided ABFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this package.  The
CUDA library never imports it, and it imports nothing from the CUDA library.

Contents
--------
* :func:`fft`, :func:`ifft` -- plain FP64 radix-2 DIT FFT written in C
  (``tfft_oracle.c``), forward unnormalised, inverse scaled by 1/N, exactly the
  DFT of TurboFFT Section II.
* :func:`dft_naive` -- the O(N^2) definition summed in long double (pins only).
* :func:`fft_faulty` -- the radix-2 FFT of one signal run in FP32 or FP64 with
  one bit of one intermediate value flipped (Section II-A fault model).
* :mod:`oracle.abft` -- the two-sided checksum scheme of Section III
  (encode, detect, locate, correct), written in numpy FP64.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(brute force, closed forms, invariants, numpy's FFT); the detection threshold
constant kappa has no printed value in the paper and is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile ``tfft_oracle.c`` into ``liboracle.so`` beside it (gcc, -O2,
    no FMA contraction so FP32 emulation rounds every operation)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_lib()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_fft.argtypes = [P, I64, I64, ctypes.c_int]
            lib.oracle_dft_naive.argtypes = [P, P, I64, I64, ctypes.c_int]
            lib.oracle_fft_faulty.argtypes = [P, P, I64, ctypes.c_int, ctypes.c_int,
                                              I64, ctypes.c_int, ctypes.c_int]
            for f in (lib.oracle_fft, lib.oracle_dft_naive, lib.oracle_fft_faulty):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _transform(x, sign: int) -> np.ndarray:
    z = _as_c128(x).copy()
    n = z.shape[-1]
    batch = z.size // n if n else 0
    if _load().oracle_fft(z.ctypes.data, n, batch, sign) != 0:
        raise ValueError(f"oracle_fft rejected n={n} batch={batch}")
    return z


def fft(x) -> np.ndarray:
    """Forward DFT along the last axis, y_j = sum_n x_n e^{-2 pi i jn/N}
    (Section II), FP64, N a power of two."""
    return _transform(x, -1)


def ifft(y) -> np.ndarray:
    """Inverse DFT along the last axis, x_j = (1/N) sum_n y_n e^{+2 pi i jn/N}
    (Section II), FP64, N a power of two."""
    return _transform(y, +1)


def dft_naive(x, sign: int = -1) -> np.ndarray:
    """The DFT by its definition (Section II), summed in long double; any N."""
    x = _as_c128(x)
    n = x.shape[-1]
    y = np.empty_like(x)
    if _load().oracle_dft_naive(x.ctypes.data, y.ctypes.data, n, x.size // n, sign) != 0:
        raise ValueError("oracle_dft_naive rejected its arguments")
    return y


def dft_bins(x, bins, sign: int = -1, chunk: int = 1 << 22) -> np.ndarray:
    """Selected outputs y_k = sum_n x_n e^{sign 2 pi i n k / N} of one signal
    by the definition (Section II), FP64.  The phase index n k is reduced
    modulo N in exact integer arithmetic before the angle is formed, so the
    twiddles carry no error from a large argument.  For spot checks of
    transforms too long for the full oracle."""
    x = _as_c128(np.asarray(x).reshape(-1))
    n = x.size
    out = np.zeros(len(bins), dtype=np.complex128)
    for j, k in enumerate(bins):
        k = int(k) % n
        acc = 0j
        for s0 in range(0, n, chunk):
            idx = np.arange(s0, min(n, s0 + chunk), dtype=np.int64)
            m = (idx * k) % n
            ang = (2.0 * np.pi / n) * m.astype(np.float64)
            acc += np.sum(x[s0:s0 + idx.size] * (np.cos(ang) + sign * 1j * np.sin(ang)))
        out[j] = acc
    return out


def fft_faulty(x, prec: int, stage: int = -2, elem: int = 0, comp: int = 0,
               bit: int = -1) -> np.ndarray:
    """Forward radix-2 FFT of ONE signal in FP32 (prec=32) or FP64 (prec=64)
    with bit ``bit`` of the real (comp=0) / imaginary (comp=1) part of working
    element ``elem`` flipped after stage ``stage`` (-1 = the loaded input,
    log2(N)-1 = the output).  bit=-1 gives a clean run in that precision.
    Emulates the Section II-A single-event-upset fault model on the CPU."""
    x = _as_c128(x)
    if x.ndim != 1:
        raise ValueError("fft_faulty takes one signal")
    y = np.empty_like(x)
    if bit < 0:
        stage = 0
    rc = _load().oracle_fft_faulty(x.ctypes.data, y.ctypes.data, x.shape[0], prec,
                                   stage, elem, comp, bit)
    if rc != 0:
        raise ValueError("oracle_fft_faulty rejected its arguments")
    return y


from . import abft  # noqa: E402,F401  (re-export the checksum scheme)
