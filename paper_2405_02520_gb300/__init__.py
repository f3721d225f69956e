"""Python binding of the GB300 fault-tolerant batched FFT (``libtfft.so``).

Argument marshalling only: every step of the transform, the checksum encode,
verification and correction runs in the library's CUDA kernels.  The names
mirror the C ABI of ``include/tfft.h``; tensors are accepted wherever the C
function takes a device pointer (their ``data_ptr()`` is passed) and torch
streams wherever it takes a ``cudaStream_t``.

There is no CPU fallback: if ``libtfft.so`` cannot be loaded (and cannot be
built because nvcc is absent) importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

from . import build as _build

TFFT_C64, TFFT_C128 = 0, 1
TFFT_ABFT_OFF, TFFT_ABFT_ONE_SIDED, TFFT_ABFT_TWO_SIDED = 0, 1, 2
TFFT_R_SIGNED_WANG, TFFT_R_WANG = 0, 1
TFFT_FORWARD, TFFT_INVERSE = 0, 1
TFFT_PREC_FP32, TFFT_PREC_TF32X3, TFFT_PREC_TF32, TFFT_PREC_BF16X3 = 0, 1, 2, 3
TFFT_RAGGED_AUTOTUNE, TFFT_RAGGED_STAGED, TFFT_RAGGED_PERSISTENT = 1, 2, 4
TFFT_FAULT_NONE, TFFT_FAULT_BITFLIP, TFFT_FAULT_SCALE, TFFT_FAULT_ADD, TFFT_FAULT_ADD_PAIR = 0, 1, 2, 3, 4
TIMING_KINDS = ("first_pass", "middle_pass", "last_pass", "single_pass", "verify", "correction")

_lock = threading.Lock()
_lib = None


class TfftError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().tfft_error_string(code).decode() if _lib is not None else str(code)
        extra = ""
        if code == -3 and _lib is not None:
            extra = f" (cudaError {_lib.tfft_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{code}]{extra}")


class PlanOpts(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("batch", ctypes.c_int64), ("dtype", ctypes.c_int),
                ("abft_mode", ctypes.c_int), ("group", ctypes.c_int), ("kappa", ctypes.c_double),
                ("detect_only", ctypes.c_int), ("max_faults", ctypes.c_int),
                ("force_passes", ctypes.c_int), ("checksum_vector", ctypes.c_int),
                ("checksum_seed", ctypes.c_uint64), ("direction", ctypes.c_int), ("normalize", ctypes.c_int),
                ("precision", ctypes.c_int), ("wait_polls", ctypes.c_int), ("first_pass_log2", ctypes.c_int),
                ("tile_threads", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("detected", ctypes.c_int64), ("corrected", ctypes.c_int64),
                ("recomputed", ctypes.c_int64), ("uncorrectable", ctypes.c_int64),
                ("execs", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("max_clean_ratio", ctypes.c_double)]


class FaultEvent(ctypes.Structure):
    _fields_ = [("exec_index", ctypes.c_int64), ("group", ctypes.c_int64), ("signal", ctypes.c_int64),
                ("action", ctypes.c_int32), ("nonfinite", ctypes.c_int32), ("residual", ctypes.c_double),
                ("tau", ctypes.c_double), ("q_re", ctypes.c_double), ("q_im", ctypes.c_double)]


class Fault(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("pass_", ctypes.c_int), ("stage", ctypes.c_int),
                ("bit", ctypes.c_int), ("signal", ctypes.c_int64), ("line", ctypes.c_int64),
                ("index", ctypes.c_int64), ("factor", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("first_pass_log2", ctypes.c_int), ("tile_threads", ctypes.c_int),
                ("candidates", ctypes.c_int), ("ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("batch", ctypes.c_int64), ("dtype", ctypes.c_int),
                ("abft_mode", ctypes.c_int), ("passes", ctypes.c_int), ("nsub", ctypes.c_int * 3),
                ("stages", ctypes.c_int * 3), ("lines_per_tile", ctypes.c_int * 3),
                ("lines_per_signal", ctypes.c_int64 * 3), ("group", ctypes.c_int),
                ("max_faults", ctypes.c_int), ("kappa", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64), ("launches_per_exec", ctypes.c_int),
                ("checksum_vector", ctypes.c_int), ("checksum_seed", ctypes.c_uint64),
                ("direction", ctypes.c_int), ("normalize", ctypes.c_int), ("precision", ctypes.c_int),
                ("tile_threads", ctypes.c_int * 3), ("tuned", ctypes.c_int)]


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            L = ctypes.CDLL(path)
            P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            PP = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "tfft_plan": [PP, I64, I64, I, I],
                "tfft_plan_ex": [PP, ctypes.POINTER(PlanOpts)],
                "tfft_exec": [P, P, P, P],
                "tfft_exec_host": [P, P, P, P],
                "tfft_report": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
                "tfft_report_ex": [P, ctypes.POINTER(Stats)],
                "tfft_reset_counters": [P],
                "tfft_fault_log": [P, ctypes.POINTER(FaultEvent), I, ctypes.POINTER(I64)],
                "tfft_set_fault": [P, ctypes.POINTER(Fault)],
                "tfft_plan_info": [P, ctypes.POINTER(Info)],
                "tfft_set_timing": [P, I],
                "tfft_timing": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I],
                "tfft_destroy": [P],
                "tfft_exec_noalloc": [I64, I64, P, P, P],
                "tfft_ragged_plan": [PP, ctypes.POINTER(I64), I64, I, I, I],
                "tfft_ragged_exec": [P, P, P, P],
                "tfft_ragged_report": [P, ctypes.POINTER(Stats)],
                "tfft_ragged_set_fault": [P, I64, ctypes.POINTER(Fault)],
                "tfft_ragged_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I),
                                     ctypes.POINTER(I), I64],
                "tfft_ragged_destroy": [P],
                "tfft_ragged_families": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
                "tfft_tc_selftest": [P, P, P, I],
                "tfft_measure_fma_peak": [I, I, ctypes.POINTER(ctypes.c_double)],
                "tfft_autotune": [ctypes.POINTER(PlanOpts), P, P, P, I, ctypes.POINTER(TuneResult)],
                "tfft_tune_lookup": [ctypes.POINTER(PlanOpts), ctypes.POINTER(PlanOpts)],
                "tfft_tune_clear": [],
                "tfft_error_string": [I],
                "tfft_last_cuda_error": [],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name == "tfft_error_string" else ctypes.c_int
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError(f"not a stream: {type(s)}")


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise TfftError(rc, where)


# ------------------------------------------------------------ C-ABI names
def tfft_plan(n: int, batch: int, dtype: int = TFFT_C64, abft_mode: int = TFFT_ABFT_TWO_SIDED) -> int:
    h = ctypes.c_void_p()
    _check(lib().tfft_plan(ctypes.byref(h), n, batch, dtype, abft_mode), "tfft_plan")
    return h.value


def tfft_plan_ex(n: int, batch: int, dtype: int = TFFT_C64, abft_mode: int = TFFT_ABFT_TWO_SIDED,
                 group: int = 0, kappa: float = 0.0, detect_only: bool = False, max_faults: int = 0,
                 force_passes: int = 0, checksum_vector: int = TFFT_R_SIGNED_WANG, checksum_seed: int = 0,
                 direction: int = TFFT_FORWARD, normalize: bool = False, precision: int = TFFT_PREC_FP32,
                 wait_polls: int = 0, first_pass_log2: int = 0, tile_threads: int = 0) -> int:
    o = PlanOpts(n, batch, dtype, abft_mode, group, kappa, int(detect_only), max_faults, force_passes,
                 checksum_vector, checksum_seed, direction, int(normalize), precision, wait_polls,
                 first_pass_log2, tile_threads)
    h = ctypes.c_void_p()
    _check(lib().tfft_plan_ex(ctypes.byref(h), ctypes.byref(o)), "tfft_plan_ex")
    return h.value


def tfft_exec(plan: int, x, y, stream=None) -> None:
    _check(lib().tfft_exec(plan, _ptr(x), _ptr(y), _stream(stream)), "tfft_exec")


def tfft_exec_host(plan: int, host_in, host_out, stream=None) -> None:
    _check(lib().tfft_exec_host(plan, _ptr(host_in), _ptr(host_out), _stream(stream)), "tfft_exec_host")


def tfft_report(plan: int) -> tuple[int, int]:
    d, c = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().tfft_report(plan, ctypes.byref(d), ctypes.byref(c)), "tfft_report")
    return d.value, c.value


def tfft_report_ex(plan: int) -> dict:
    s = Stats()
    _check(lib().tfft_report_ex(plan, ctypes.byref(s)), "tfft_report_ex")
    return {f: getattr(s, f) for f, _ in Stats._fields_}


def tfft_reset_counters(plan: int) -> None:
    _check(lib().tfft_reset_counters(plan), "tfft_reset_counters")


def tfft_fault_log(plan: int, capacity: int = 1024) -> tuple[list, int]:
    arr = (FaultEvent * max(1, capacity))()
    tot = ctypes.c_int64()
    _check(lib().tfft_fault_log(plan, arr, capacity, ctypes.byref(tot)), "tfft_fault_log")
    n = min(capacity, tot.value)
    return [{f: getattr(arr[k], f) for f, _ in FaultEvent._fields_} for k in range(n)], tot.value


def tfft_set_fault(plan: int, mode: int, pass_: int = 0, stage: int = -1, signal: int = 0,
                   line: int = 0, index: int = 0, bit: int = 0, factor: float = 0.0) -> None:
    f = Fault(mode, pass_, stage, bit, signal, line, index, factor)
    _check(lib().tfft_set_fault(plan, ctypes.byref(f)), "tfft_set_fault")


def tfft_plan_info(plan: int) -> dict:
    i = Info()
    _check(lib().tfft_plan_info(plan, ctypes.byref(i)), "tfft_plan_info")
    out = {}
    for f, _ in Info._fields_:
        v = getattr(i, f)
        out[f] = list(v) if not isinstance(v, (int, float)) else v
    return out


def tfft_set_timing(plan: int, enable: bool) -> None:
    _check(lib().tfft_set_timing(plan, int(enable)), "tfft_set_timing")


def tfft_timing(plan: int) -> dict:
    k = len(TIMING_KINDS)
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_int64 * k)()
    _check(lib().tfft_timing(plan, ms, cnt, k), "tfft_timing")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(TIMING_KINDS)}


def tfft_destroy(plan: int) -> None:
    _check(lib().tfft_destroy(plan), "tfft_destroy")


class Ragged:
    """A ragged batch: signals of different power-of-two lengths packed back
    to back (see include/tfft.h, tfft_ragged_*)."""

    def __init__(self, lengths, dtype: int = TFFT_C64, abft_mode: int = TFFT_ABFT_TWO_SIDED,
                 autotune: bool = True, staged: bool = False, persistent: bool = False):
        arr = (ctypes.c_int64 * len(lengths))(*[int(v) for v in lengths])
        h = ctypes.c_void_p()
        flags = ((TFFT_RAGGED_AUTOTUNE if autotune else 0) | (TFFT_RAGGED_STAGED if staged else 0)
                 | (TFFT_RAGGED_PERSISTENT if persistent else 0))
        _check(lib().tfft_ragged_plan(ctypes.byref(h), arr, len(lengths), dtype, abft_mode, flags),
               "tfft_ragged_plan")
        self.handle = h.value
        self.lengths = [int(v) for v in lengths]

    def exec(self, x, y, stream=None) -> None:
        _check(lib().tfft_ragged_exec(self.handle, _ptr(x), _ptr(y), _stream(stream)), "tfft_ragged_exec")

    def report(self) -> dict:
        s = Stats()
        _check(lib().tfft_ragged_report(self.handle, ctypes.byref(s)), "tfft_ragged_report")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def set_fault(self, signal: int, mode: int, pass_: int = 0, stage: int = -1, line: int = 0, index: int = 0,
                  bit: int = 0, factor: float = 0.0) -> None:
        f = Fault(mode, pass_, stage, bit, 0, line, index, factor)
        _check(lib().tfft_ragged_set_fault(self.handle, signal, ctypes.byref(f)), "tfft_ragged_set_fault")

    def _info(self):
        nb = ctypes.c_int64()
        _check(lib().tfft_ragged_info(self.handle, ctypes.byref(nb), None, None, None, 0), "tfft_ragged_info")
        ln = (ctypes.c_int64 * nb.value)()
        ps = (ctypes.c_int * nb.value)()
        dr = (ctypes.c_int * nb.value)()
        _check(lib().tfft_ragged_info(self.handle, ctypes.byref(nb), ln, ps, dr, nb.value), "tfft_ragged_info")
        return [(ln[k], ps[k], dr[k]) for k in range(nb.value)]

    def info(self) -> list:
        """[(length, passes)] per bucket, longest first."""
        return [(n, p) for n, p, _ in self._info()]

    def layout(self) -> dict:
        """{length: True if the bucket is addressed in place, False if staged}."""
        return {n: bool(d) for n, _, d in self._info()}

    def families(self) -> tuple[int, int]:
        """(pass families, buckets run in them) of the persistent form."""
        f, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tfft_ragged_families(self.handle, ctypes.byref(f), ctypes.byref(b)), "tfft_ragged_families")
        return f.value, b.value

    def destroy(self) -> None:
        if self.handle:
            _check(lib().tfft_ragged_destroy(self.handle), "tfft_ragged_destroy")
            self.handle = None


def tfft_tc_selftest(a, bt, d, terms: int) -> None:
    """D = A B for one 128 x 32 x 32 tile on the tensor cores (see include/tfft.h)."""
    _check(lib().tfft_tc_selftest(_ptr(a), _ptr(bt), _ptr(d), terms), "tfft_tc_selftest")


def tfft_exec_noalloc(n: int, batch: int, x, y, stream=None) -> None:
    """Allocation-free two-pass complex64 transform (see include/tfft.h)."""
    _check(lib().tfft_exec_noalloc(n, batch, _ptr(x), _ptr(y), _stream(stream)), "tfft_exec_noalloc")


def tfft_measure_fma_peak(fp64: bool, iters: int) -> float:
    """Measured multiply-add throughput of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(lib().tfft_measure_fma_peak(int(bool(fp64)), iters, ctypes.byref(v)), "tfft_measure_fma_peak")
    return v.value


def _opts(n: int, batch: int, dtype: int, abft_mode: int, **kw) -> PlanOpts:
    o = PlanOpts()
    o.n, o.batch, o.dtype, o.abft_mode = n, batch, dtype, abft_mode
    for k, v in kw.items():
        setattr(o, k, int(v) if not isinstance(v, float) else v)
    return o


def tfft_autotune(n: int, batch: int, dtype: int, abft_mode: int, x, y, stream=None, reps: int = 5,
                  **opts) -> dict:
    """Times every admissible pass configuration on x -> y and records the
    fastest in the autotuner's table (see include/tfft.h); returns it."""
    o = _opts(n, batch, dtype, abft_mode, **opts)
    r = TuneResult()
    _check(lib().tfft_autotune(ctypes.byref(o), _ptr(x), _ptr(y), _stream(stream), reps, ctypes.byref(r)),
           "tfft_autotune")
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def tfft_tune_lookup(n: int, batch: int, dtype: int, abft_mode: int, **opts):
    """The table's configuration for these options as (passes, first_pass_log2,
    tile_threads), or None."""
    o = _opts(n, batch, dtype, abft_mode, **opts)
    t = PlanOpts()
    rc = lib().tfft_tune_lookup(ctypes.byref(o), ctypes.byref(t))
    _check(min(rc, 0), "tfft_tune_lookup")
    return (t.force_passes, t.first_pass_log2, t.tile_threads) if rc == 1 else None


def tfft_tune_clear() -> None:
    _check(lib().tfft_tune_clear(), "tfft_tune_clear")


def tfft_error_string(code: int) -> str:
    return lib().tfft_error_string(code).decode()


@dataclass
class Plan:
    """RAII holder of a plan handle (``with Plan(...) as p: p.exec(x, y)``)."""
    n: int
    batch: int
    dtype: int = TFFT_C64
    abft_mode: int = TFFT_ABFT_TWO_SIDED
    group: int = 0
    kappa: float = 0.0
    detect_only: bool = False
    max_faults: int = 0
    force_passes: int = 0
    checksum_vector: int = TFFT_R_SIGNED_WANG
    checksum_seed: int = 0
    direction: int = TFFT_FORWARD
    normalize: bool = False
    precision: int = TFFT_PREC_FP32

    def __post_init__(self):
        self.handle = tfft_plan_ex(self.n, self.batch, self.dtype, self.abft_mode, self.group,
                                   self.kappa, self.detect_only, self.max_faults, self.force_passes,
                                   self.checksum_vector, self.checksum_seed, self.direction, self.normalize,
                                   self.precision)

    def exec(self, x, y, stream=None):
        tfft_exec(self.handle, x, y, stream)

    def report(self):
        return tfft_report_ex(self.handle)

    def info(self):
        return tfft_plan_info(self.handle)

    def destroy(self):
        if getattr(self, "handle", None):
            tfft_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
