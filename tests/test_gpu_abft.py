"""Two-sided ABFT on the GPU: detection, location and correction of injected
faults (Section II-A fault model, Section III scheme), and no false alarms."""
import numpy as np
import pytest

import oracle
from oracle import abft as oabft
import paper_2405_02520_gb300 as t
from paper_2405_02520_gb300.inputs import normal_batch, uniform_batch
from tests.gpu_util import oracle_fft, rel_err_rows, run_gpu, tol

pytestmark = pytest.mark.gpu


def test_config1_scaled_output_element_detected_located_corrected():
    """N = 1024, batch 256, U[-1,1) from seed 0; one output element of one
    signal multiplied by 1 + 1e-2, site drawn from seed 1."""
    n, batch = 1024, 256
    x = uniform_batch(n, batch, seed=0)
    rng = np.random.default_rng(1)
    sig, idx = int(rng.integers(batch)), int(rng.integers(n))
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=0, stage=info["stages"][0] - 1, signal=sig,
                 line=0, index=idx, factor=1.0 + 1e-2)
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    ref = oracle_fft(x)
    assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (1, 1)
    ev, total = t.tfft_fault_log(plan)
    assert total == 1 and ev[0]["signal"] == sig and ev[0]["action"] == 1
    assert abs(ev[0]["q_re"] - (sig % info["group"] + 1)) < 0.05
    t.tfft_destroy(plan)

    # the same fault left uncorrected is harmful, and the oracle's own
    # checksum test names the same group and signal
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, detect_only=True)
    yf, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    assert rel_err_rows(yf[sig:sig + 1], ref[sig:sig + 1])[0] > tol(n, t.TFFT_C64)
    kind = "signed_wang" if info["checksum_vector"] == t.TFFT_R_SIGNED_WANG else "wang"
    res = oabft.run(x, yf, group=info["group"], u=2.0 ** -24, kappa=info["kappa"], kind=kind,
                    seed=info["checksum_seed"])
    assert res.located == {sig // info["group"]: sig}
    assert t.tfft_report(plan)[0] == 1
    t.tfft_destroy(plan)


def _site(info, rng, passes=None):
    p = int(rng.integers(info["passes"])) if passes is None else passes
    stage = int(rng.integers(-1, info["stages"][p]))
    line = int(rng.integers(info["lines_per_signal"][p]))
    index = int(rng.integers(info["nsub"][p]))
    return p, stage, line, index


@pytest.mark.parametrize("log2n,batch", [(10, 64), (16, 8), (19, 6), (20, 4)])
def test_large_bitflips_every_pass_corrected(log2n, batch):
    """High exponent/mantissa bit flips (bits 26..30 of the real part) at
    random (pass, stage, signal, element): detected, named, corrected."""
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=40 + log2n)
    ref = oracle_fft(x)
    rng = np.random.default_rng(log2n)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    expect = 0
    for trial in range(12):
        p, stage, line, index = _site(info, rng)
        sig = int(rng.integers(batch))
        bit = int(rng.integers(26, 31))
        fault = dict(mode=t.TFFT_FAULT_BITFLIP, pass_=p, stage=stage, signal=sig, line=line,
                     index=index, bit=bit)
        y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
        err = rel_err_rows(y, ref)
        assert err.max() <= tol(n, t.TFFT_C64), (trial, fault, err.max())
        d, c = t.tfft_report(plan)
        expect += 1
        assert d == expect and c == expect, (trial, fault, d, c)
    t.tfft_destroy(plan)


def test_nonfinite_fault_located_and_corrected():
    n, batch = 4096, 32
    x = uniform_batch(n, batch, seed=9)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    fault = dict(mode=t.TFFT_FAULT_SCALE, pass_=0, stage=1, signal=21, line=0, index=77,
                 factor=float("inf"))
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    assert np.all(np.isfinite(y))
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    ev, _ = t.tfft_fault_log(plan)
    assert ev[-1]["signal"] == 21 and ev[-1]["nonfinite"] == 1
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n", [10, 16, 19])
def test_two_faults_in_a_group_fall_back_to_recompute(log2n):
    n = 1 << log2n
    batch = 40
    x = uniform_batch(n, batch, seed=11)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    fault = dict(mode=t.TFFT_FAULT_ADD_PAIR, pass_=info["passes"] - 1,
                 stage=info["stages"][info["passes"] - 1] - 1, signal=18, line=0, index=5,
                 factor=3.0)
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
    assert rel_err_rows(y, oracle_fft(x)).max() <= tol(n, t.TFFT_C64)
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 1 and st["recomputed"] == 1, st
    t.tfft_destroy(plan)


def test_c128_one_fault_per_launch():
    """complex128, N = 2^12 x 2^14 reduced to 256 signals: one fault per
    launch, corrected to 1e-14 log2 N."""
    n, batch = 1 << 12, 256
    x = normal_batch(n, batch, seed=3)
    ref = oracle_fft(x)
    plan = t.tfft_plan(n, batch, t.TFFT_C128, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    rng = np.random.default_rng(33)
    for k in range(6):
        p, stage, line, index = _site(info, rng)
        fault = dict(mode=t.TFFT_FAULT_BITFLIP, pass_=p, stage=stage, signal=int(rng.integers(batch)),
                     line=line, index=index, bit=int(rng.integers(56, 63)))
        y, _ = run_gpu(x, t.TFFT_C128, plan=plan, fault=fault)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C128), (k, fault)
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 6 and st["corrected"] + st["recomputed"] == 6
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n,batch,launches", [(10, 256, 300), (16, 64, 50), (20, 16, 20)])
def test_no_false_positives_on_clean_launches(log2n, batch, launches):
    import torch
    n = 1 << log2n
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    y = torch.empty(batch, n, dtype=torch.complex64, device="cuda")
    for s in range(launches):
        x = torch.from_numpy(uniform_batch(n, batch, seed=10000 + s)).cuda()
        t.tfft_exec(plan, x, y, torch.cuda.current_stream())
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n,batch", [(10, 64), (16, 20)])
def test_correction_graph_replayed_with_faults(log2n, batch):
    """The same buffers exec'd again and again (verification and correction
    replayed from the plan's graph; N = 1024 x 64 is a fused plan, whose
    kernel corrects in its last block instead): clean execs stay clean, a
    located fault is corrected, two faults in one group are recomputed, and
    later clean execs are clean."""
    import torch
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=5100 + log2n)
    ref = oracle_fft(x)
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)
    s = torch.cuda.current_stream()

    def run():
        t.tfft_exec(plan, xt, yt, s)
        torch.cuda.synchronize()
        assert rel_err_rows(yt.cpu().numpy(), ref).max() <= tol(n, t.TFFT_C64)

    for _ in range(3):
        run()
    assert t.tfft_report(plan) == (0, 0)
    p = info["passes"] - 1
    t.tfft_set_fault(plan, mode=t.TFFT_FAULT_SCALE, pass_=p, stage=info["stages"][p] - 1, signal=batch - 5,
                     line=0, index=7, factor=1.5)
    run()
    assert t.tfft_report(plan) == (1, 1)
    t.tfft_set_fault(plan, mode=t.TFFT_FAULT_ADD_PAIR, pass_=p, stage=info["stages"][p] - 1, signal=3, line=0,
                     index=5, factor=3.0)
    run()
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 2 and st["corrected"] == 1 and st["recomputed"] == 1, st
    for _ in range(2):
        run()
    assert t.tfft_report_ex(plan)["detected"] == 2
    t.tfft_destroy(plan)


@pytest.mark.parametrize("log2n,batch", [(10, 64), (14, 32)])
def test_plain_wang_vector_parity_and_fault(log2n, batch):
    """The paper's own left vector e_Wang (r_k = w3^k, w in closed form):
    clean output within the tolerance with no false alarm; a scaled output
    element and a large input-side flip are each detected, named and
    corrected, and the oracle's per-signal scheme with kind "wang" flags and
    names the same signal on the uncorrected output.  (The input-side flip is
    seen through |w_n| / sqrt(N) of its size, a few group thresholds only:
    the group quotient alone is too noisy to name its signal.)"""
    n = 1 << log2n
    x = uniform_batch(n, batch, seed=600 + log2n)
    ref = oracle_fft(x)
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, checksum_vector=t.TFFT_R_WANG)
    info = t.tfft_plan_info(plan)
    assert info["checksum_vector"] == t.TFFT_R_WANG
    y, _ = run_gpu(x, t.TFFT_C64, plan=plan)
    assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64)
    assert t.tfft_report(plan) == (0, 0)
    last = info["passes"] - 1
    faults = [dict(mode=t.TFFT_FAULT_SCALE, pass_=last, stage=info["stages"][last] - 1, signal=batch // 3,
                   line=0, index=5, factor=1.0 + 1e-2),
              dict(mode=t.TFFT_FAULT_BITFLIP, pass_=0, stage=-1, signal=batch - 2,
                   line=min(1, info["lines_per_signal"][0] - 1), index=7, bit=29)]
    for k, fault in enumerate(faults):
        y, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
        assert rel_err_rows(y, ref).max() <= tol(n, t.TFFT_C64), fault
        assert t.tfft_report(plan) == (k + 1, k + 1)
        ev, _ = t.tfft_fault_log(plan, 1)
        assert ev[-1]["signal"] == fault["signal"]
    t.tfft_destroy(plan)
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, checksum_vector=t.TFFT_R_WANG,
                          detect_only=True)
    for fault in faults:
        yf, _ = run_gpu(x, t.TFFT_C64, plan=plan, fault=fault)
        res = oabft.run(x, yf, group=info["group"], u=2.0 ** -24, kappa=info["kappa"], kind="wang",
                        per_signal=True)
        assert res.located == {fault["signal"] // info["group"]: fault["signal"]}
    t.tfft_destroy(plan)


@pytest.mark.parametrize("dtype", [t.TFFT_C64, t.TFFT_C128])
def test_fused_exec_is_one_launch_and_corrects_in_its_kernel(dtype):
    """A single-pass plan of few checksum groups (N = 1024, batch 256: 16
    groups) runs an exec as one kernel whose last block verifies and corrects:
    a huge input-side flip (located: W c1 minus the other signals' outputs),
    two faults in one group (not locatable: the group recomputed in the
    block), each exec one launch, every output within the tolerance."""
    n, batch = 1024, 256
    x = uniform_batch(n, batch, seed=77)
    if dtype == t.TFFT_C128:
        x = x.astype(np.complex128)
    ref = oracle_fft(x)
    plan = t.tfft_plan(n, batch, dtype, t.TFFT_ABFT_TWO_SIDED)
    info = t.tfft_plan_info(plan)
    assert info["passes"] == 1 and info["launches_per_exec"] == 1
    y, _ = run_gpu(x, dtype, plan=plan)
    assert rel_err_rows(y, ref).max() <= tol(n, dtype)
    assert t.tfft_report(plan) == (0, 0)
    bit = 30 if dtype == t.TFFT_C64 else 62
    faults = [dict(mode=t.TFFT_FAULT_BITFLIP, pass_=0, stage=-1, signal=200, line=0, index=9, bit=bit),
              dict(mode=t.TFFT_FAULT_ADD_PAIR, pass_=0, stage=info["stages"][0] - 1, signal=35, line=0, index=5,
                   factor=3.0)]
    for k, fault in enumerate(faults):
        before = t.tfft_report_ex(plan)["launches"]
        y, _ = run_gpu(x, dtype, plan=plan, fault=fault)
        assert t.tfft_report_ex(plan)["launches"] == before + 1
        assert rel_err_rows(y, ref).max() <= tol(n, dtype), fault
    st = t.tfft_report_ex(plan)
    assert st["detected"] == 2 and st["corrected"] == 1 and st["recomputed"] == 1, st
    ev, total = t.tfft_fault_log(plan)
    assert total == 2 and ev[0]["signal"] == 200 and ev[0]["action"] == 1 and ev[1]["action"] == 2
    t.tfft_destroy(plan)


def test_back_to_back_fused_execs_overlap_safely():
    """Eight fused execs (N = 1024, batch 128) issued back to back on one
    stream with no synchronisation between them, each on its own buffers
    (each kernel may start its set-up while the one before it verifies and
    corrects): a fault in the fifth is corrected there, and every output
    matches the oracle."""
    import torch
    n, batch = 1024, 128
    xs = [uniform_batch(n, batch, seed=880 + i) for i in range(8)]
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    assert t.tfft_plan_info(plan)["launches_per_exec"] == 1
    xt = [torch.from_numpy(x).cuda() for x in xs]
    yt = [torch.empty_like(x) for x in xt]
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for i in range(8):
        if i == 4:
            t.tfft_set_fault(plan, mode=t.TFFT_FAULT_SCALE, pass_=0, stage=0, signal=77, line=0, index=300,
                             factor=1.25)
        t.tfft_exec(plan, xt[i], yt[i], s)
    torch.cuda.synchronize()
    for i in range(8):
        assert rel_err_rows(yt[i].cpu().numpy(), oracle_fft(xs[i])).max() <= tol(n, t.TFFT_C64), i
    assert t.tfft_report(plan) == (1, 1)
    ev, _ = t.tfft_fault_log(plan)
    assert ev[-1]["signal"] == 77 and ev[-1]["exec_index"] == 4
    t.tfft_destroy(plan)


def test_fused_exec_after_a_kernel_that_writes_its_input():
    """A fused exec launched right after another kernel on the stream that
    rewrites its input buffer (an elementwise kernel) transforms the new input:
    the exec's kernel waits for the kernel before it before it loads a tile,
    whatever that kernel is."""
    import torch
    n, batch = 1024, 64
    xs = [uniform_batch(n, batch, seed=990 + i) for i in range(6)]
    src = [torch.from_numpy(x).cuda() for x in xs]
    xt = torch.empty_like(src[0])
    yt = [torch.empty_like(xt) for _ in xs]
    plan = t.tfft_plan(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    assert t.tfft_plan_info(plan)["launches_per_exec"] == 1
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for i in range(6):
        torch.mul(src[i], 1.0, out=xt)
        t.tfft_exec(plan, xt, yt[i], s)
    torch.cuda.synchronize()
    for i in range(6):
        assert rel_err_rows(yt[i].cpu().numpy(), oracle_fft(xs[i])).max() <= tol(n, t.TFFT_C64), i
    assert t.tfft_report(plan) == (0, 0)
    t.tfft_destroy(plan)
