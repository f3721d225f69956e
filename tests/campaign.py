"""Fault-injection campaign on the GPU (TurboFFT Section II-A fault model and
the Section V-C protocol): random signal, pass, stage, element and bit; each
fault is run once with correction disabled, to classify it as harmful or benign
against the FP64 oracle (harmful = the uncorrected output of the faulty signal
misses the tolerance), and once with correction on.

Usage (on a GPU):  python tests/campaign.py --log2n 10 --batch 64 --faults 200
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_2405_02520_gb300 as t  # noqa: E402
from paper_2405_02520_gb300.inputs import normal_batch, uniform_batch  # noqa: E402


def tol(n, dtype):
    return (2e-6 if dtype == t.TFFT_C64 else 1e-14) * max(1, int(np.log2(n)))


def run_campaign(n, batch, dtype=t.TFFT_C64, faults=100, seed=0, bits=None, kappa=0.0,
                 vector=t.TFFT_R_SIGNED_WANG, mode=t.TFFT_FAULT_BITFLIP):
    """`faults` single-fault execs at random sites.  Each fault runs twice:
    with correction off (detect only), to classify it against the oracle, and
    with correction on.  The oracle's FP64 transform of the batch is computed
    once on the host and kept on the device, where each exec's per-signal
    relative L2 error against it is formed (only those numbers come back)."""
    import torch
    w = 32 if dtype == t.TFFT_C64 else 64
    x = (uniform_batch(n, batch, seed=seed) if dtype == t.TFFT_C64
         else normal_batch(n, batch, seed=seed))
    ref = torch.from_numpy(oracle.fft(x.astype(np.complex128))).cuda()
    ref_norm = torch.linalg.vector_norm(ref, dim=1)
    xt = torch.from_numpy(x).cuda()
    yt = torch.empty_like(xt)

    def row_errors():
        with torch.no_grad():
            e = torch.linalg.vector_norm(yt.to(torch.complex128) - ref, dim=1) / ref_norm
        e = e.cpu().numpy()
        return np.where(np.isfinite(e), e, np.inf)

    plans = {flag: t.tfft_plan_ex(n, batch, dtype, t.TFFT_ABFT_TWO_SIDED, kappa=kappa,
                                  detect_only=flag, checksum_vector=vector)
             for flag in (True, False)}
    info = t.tfft_plan_info(plans[False])
    rng = np.random.default_rng(1000 + seed)
    out = {"n": n, "batch": batch, "dtype": "c64" if dtype == t.TFFT_C64 else "c128",
           "kappa": info["kappa"], "vector": "signed_wang" if vector == t.TFFT_R_SIGNED_WANG else "wang",
           "faults": 0, "harmful": 0, "harmful_detected": 0, "harmful_located": 0,
           "harmful_corrected": 0, "benign": 0, "benign_detected": 0, "benign_output_ok": 0,
           "clear": 0, "clear_detected": 0, "clear_corrected": 0, "marginal": 0, "marginal_missed": 0,
           "marginal_detected": 0, "missed": [], "by_stage": {}, "max_corrected_err": 0.0}
    tl = tol(n, dtype)
    for k in range(faults):
        p = int(rng.integers(info["passes"]))
        stage = int(rng.integers(-1, info["stages"][p]))
        line = int(rng.integers(info["lines_per_signal"][p]))
        index = int(rng.integers(info["nsub"][p]))
        sig = int(rng.integers(batch))
        bit = int(rng.integers(*(bits or (0, 2 * w))))
        site = dict(mode=mode, pass_=p, stage=stage, signal=sig, line=line, index=index, bit=bit,
                    factor=0.0)
        res = {}
        for flag in (True, False):
            plan = plans[flag]
            before = t.tfft_report_ex(plan)
            t.tfft_set_fault(plan, **site)
            t.tfft_exec(plan, xt, yt, torch.cuda.current_stream())
            torch.cuda.synchronize()
            after = t.tfft_report_ex(plan)
            ev, _ = t.tfft_fault_log(plan, 1)
            det = after["detected"] > before["detected"]
            res[flag] = (row_errors(), det, ev[-1]["signal"] if det and ev else None)
        err_unc, det, loc = res[True]
        err_cor = res[False][0]
        err = err_unc[sig]
        harmful = err > tl
        ok = bool(np.all(err_cor <= tl))
        out["max_corrected_err"] = max(out["max_corrected_err"], float(np.max(err_cor)))
        if err > 2 * tl:                  # harmful by a margin
            out["clear"] += 1
            out["clear_detected"] += det
            out["clear_corrected"] += ok
        elif harmful:                     # within a factor of two of the tolerance
            out["marginal"] += 1
            out["marginal_detected"] += det
            out["marginal_missed"] += not det
        key = f"p{p}s{stage}"
        bs = out["by_stage"].setdefault(key, [0, 0])
        out["faults"] += 1
        if harmful:
            out["harmful"] += 1
            bs[0] += 1
            out["harmful_detected"] += det
            out["harmful_located"] += (loc == sig)
            out["harmful_corrected"] += ok
            if not (det and ok and loc == sig):
                bs[1] += 1
                out["missed"].append(dict(site, err=float(err)))
        else:
            out["benign"] += 1
            out["benign_detected"] += det
            out["benign_output_ok"] += ok
    stats = t.tfft_report_ex(plans[False])
    out["max_clean_ratio"] = stats["max_clean_ratio"]
    for plan in plans.values():
        t.tfft_destroy(plan)
    return out


def clean_campaign(n, batch, launches, seed0=10000, kappa=0.0):
    """`launches` fault-free transforms of fresh seeded inputs; returns the
    detection count and the largest residual / threshold seen."""
    import torch
    from paper_2405_02520_gb300.inputs import uniform_batch_device
    plan = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, kappa=kappa)
    y = torch.empty(batch, n, dtype=torch.complex64, device="cuda")
    for s in range(launches):
        x = uniform_batch_device(n, batch, seed0 + s)
        t.tfft_exec(plan, x, y, torch.cuda.current_stream())
    st = t.tfft_report_ex(plan)
    t.tfft_destroy(plan)
    return {"n": n, "batch": batch, "launches": launches, "groups_checked": launches * ((batch + 15) // 16),
            "detected": st["detected"], "max_clean_ratio": st["max_clean_ratio"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2n", type=int, nargs="+", default=[10, 16, 20])
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--faults", type=int, default=100)
    ap.add_argument("--c128", action="store_true")
    ap.add_argument("--wang", action="store_true")
    ap.add_argument("--kappa", type=float, default=0.0)
    ap.add_argument("--clean", type=int, default=0, help="also run this many clean launches")
    a = ap.parse_args()
    for lg in a.log2n:
        n = 1 << lg
        b = a.batch or max(4, min(64, (1 << 22) // n))
        r = run_campaign(n, b, t.TFFT_C128 if a.c128 else t.TFFT_C64, a.faults, seed=lg, kappa=a.kappa,
                         vector=t.TFFT_R_WANG if a.wang else t.TFFT_R_SIGNED_WANG)
        r["missed"] = r["missed"][:5]
        print(json.dumps(r), flush=True)
        if a.clean:
            print(json.dumps(clean_campaign(n, b, a.clean, kappa=a.kappa)), flush=True)


if __name__ == "__main__":
    main()
