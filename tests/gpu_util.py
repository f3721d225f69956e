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


def run_gpu(x: np.ndarray, dtype, abft=True, plan=None, fault=None, **plan_kw):
    """Transform x (batch, n) on the GPU; returns (y, plan handle)."""
    import torch
    b, n = x.shape
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yt = torch.empty_like(xt)
    own = plan is None
    if own:
        plan = t.tfft_plan_ex(n, b, dtype, t.TFFT_ABFT_TWO_SIDED if abft else t.TFFT_ABFT_OFF, **plan_kw)
    if fault is not None:
        t.tfft_set_fault(plan, **fault)
    t.tfft_exec(plan, xt, yt, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yt.cpu().numpy(), plan


def rel_err_rows(y, ref):
    y = y.astype(np.complex128)
    num = np.linalg.norm(y - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)
    return num / den


def oracle_fft(x):
    return oracle.fft(x.astype(np.complex128))
