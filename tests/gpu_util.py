"""Helpers for the GPU tests: run the CUDA path through the C ABI on torch
device buffers and compare with the FP64 oracle."""
import numpy as np

import oracle
import paper_2405_02520_gb300 as t


def np_dtype(dtype):
    return np.complex64 if dtype == t.TFFT_C64 else np.complex128


def tol(n, dtype):
    """Relative-L2 bound per signal: 2e-6 log2 N (complex64) and
    1e-14 log2 N (complex128)."""
    lg = max(1, int(np.log2(n)))
    return (2e-6 if dtype == t.TFFT_C64 else 1e-14) * lg


# Canary guard words (the stand-in for a memory checker): every device buffer
# a test hands to the library sits between GUARD values of a fixed bit
# pattern on each side, checked after the call, so a store past either end of
# an output (or any store into an input) fails the test.
GUARD = 64                      # complex values on each side (512 or 1024 bytes: alignment kept)
CANARY = 0x7FC0DEAD             # a NaN bit pattern no transform writes


class Guarded:
    """A device tensor of `shape` and `dtype` with canary words around it."""

    def __init__(self, shape, dtype, device="cuda", fill=None):
        import torch
        if dtype is None:
            dtype = fill.dtype
        self.count = int(np.prod(shape))
        self.buf = torch.empty(self.count + 2 * GUARD, dtype=dtype, device=device)
        self.words = self.buf.view(torch.int32)
        per = self.words.numel() // (self.count + 2 * GUARD)
        self.edge = GUARD * per
        self.words[:self.edge] = CANARY
        self.words[-self.edge:] = CANARY
        self.t = self.buf[GUARD:GUARD + self.count].view(*shape)
        if fill is not None:
            self.t.copy_(fill)

    def check(self, what="buffer"):
        import torch
        lo = self.words[:self.edge]
        hi = self.words[-self.edge:]
        assert bool(torch.all(lo == CANARY)), f"{what}: store below the start of the buffer"
        assert bool(torch.all(hi == CANARY)), f"{what}: store past the end of the buffer"


def run_gpu(x: np.ndarray, dtype, abft=True, plan=None, fault=None, **plan_kw):
    """Transform x (batch, n) on the GPU; returns (y, plan handle).  The input
    and output sit between canary words, checked after the exec, and the
    input must come back unchanged."""
    import torch
    b, n = x.shape
    xh = np.ascontiguousarray(x)
    src = torch.from_numpy(xh)
    xg = Guarded((b, n), src.dtype, fill=src.cuda())
    yg = Guarded((b, n), src.dtype)
    own = plan is None
    if own:
        plan = t.tfft_plan_ex(n, b, dtype, t.TFFT_ABFT_TWO_SIDED if abft else t.TFFT_ABFT_OFF, **plan_kw)
    if fault is not None:
        t.tfft_set_fault(plan, **fault)
    t.tfft_exec(plan, xg.t, yg.t, torch.cuda.current_stream())
    torch.cuda.synchronize()
    xg.check("input"); yg.check("output")
    assert np.array_equal(xg.t.cpu().numpy(), xh), "the input was written"
    return yg.t.cpu().numpy(), plan


def rel_err_rows(y, ref):
    y = y.astype(np.complex128)
    num = np.linalg.norm(y - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)
    return num / den


def oracle_fft(x):
    return oracle.fft(x.astype(np.complex128))
