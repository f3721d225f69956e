#!/usr/bin/env python3
"""Throughput benchmark of the fault-tolerant batched FFT (one JSON line).

Workload: the batched 1-D complex-to-complex FFT, complex64, swept over
N = 2^8 .. 2^24 (powers of two) with batch = 2^28 / N, i.e. 2^28 elements
(2 GiB in, 2 GiB out) per transform, inputs i.i.d. uniform [-1, 1) in real and
imaginary parts, two-sided ABFT on.  One step = one transform of every N of
the sweep.  GFLOP/s counts 5 N log2 N flops per signal.

Reported: whole-job GFLOP/s from CUDA events over K steps (max over ranks);
the HBM roofline fraction of the dominant kernel from the library's
per-launch events over the same timed region; the ABFT overhead against the
same sweep with ABFT off; an end-to-end number through tfft_exec_host (host
buffers, copies inside the timed region); the FP64 CPU oracle timed on a
bounded sample; SM clocks sampled during the timed region.

Multi-GPU (torchrun, one process per GPU): signals are independent, so each
rank runs the whole sweep on its own GPU (weak scaling) with no collective on
the data path; only the timing is reduced (max over ranks).

--impl reference times the FP64 CPU oracle (radix-2 FFT plus the checksum
encode and verification) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP = list(range(8, 25))
TOTAL_LOG2 = 28
METRIC = "GFLOP/s (5N·log2N) and % HBM roofline with ABFT on; ABFT overhead %; vs plain FP32"
KERNEL_KINDS = ("first_pass", "middle_pass", "last_pass", "single_pass", "verify", "correction")
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend: str):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_scalar(value: float, op: str, device=None) -> float:
    """max / sum of a scalar over ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def shard_signals(batch: int, world: int, rank: int, group: int):
    """Contiguous whole-group slice of the batch for one rank (used when a
    single batch is split instead of replicated)."""
    groups = (batch + group - 1) // group
    g0 = (groups * rank) // world
    g1 = (groups * (rank + 1)) // world
    return min(batch, g0 * group), min(batch, g1 * group)


# ------------------------------------------------------------------ utils
def flops(n: int, batch: int) -> float:
    return 5.0 * n * np.log2(n) * batch if n > 1 else 0.0


def min_passes(n: int) -> int:
    """Fewest passes over HBM for an N-point complex64 transform: one tile
    holds N <= 4096, two passes of sub-transforms up to 8192 points reach
    2^26, three beyond (Section IV-A)."""
    return 1 if n <= 4096 else (2 if n <= 1 << 26 else 3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2405_02520_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind: str, elements: int):
    """DRAM bytes per launch of `kind` from the committed ncu summary, only if
    it was taken on the current kernel sources, for launches of `elements`
    values (the summary's bytes scale with the elements of a launch)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_hash") != kernel_source_hash():
            return None
        b = d.get("bytes_per_launch", {}).get(kind)
        if b is None:
            return None
        return int(round(b * elements / d.get("bench_elements_per_launch", elements)))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        power = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons,
                "samples": len(self.rows),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------- CPU oracle
_SAMPLE_INPUTS = {}


def oracle_sample(elems_per_n: int, seed: int = 0, sweep=SWEEP):
    """Time the FP64 oracle (radix-2 FFT + two-sided checksum encode and
    verification per group of 16) on max(1, elems_per_n / N) signals of
    each N.  Inputs and checksum vectors are made once per process and kept
    (host-resident, like the GPU arm's inputs in HBM); only the transform and
    the checksum work are timed.  Returns (flops, seconds, description)."""
    import oracle
    from oracle import abft
    from paper_2405_02520_gb300.inputs import uniform_batch
    tot_flops, tot_s, desc = 0.0, 0.0, []
    for lg in sweep:
        n = 1 << lg
        b = max(1, elems_per_n // n)
        key = (lg, b, seed)
        if key not in _SAMPLE_INPUTS:
            _SAMPLE_INPUTS[key] = uniform_batch(n, b, seed=seed + lg).astype(np.complex128)
        if ("rw", lg) not in _SAMPLE_INPUTS:
            _SAMPLE_INPUTS[("rw", lg)] = abft.vectors(n, "signed_wang", seed=20240502)
        x = _SAMPLE_INPUTS[key]
        r, w = _SAMPLE_INPUTS[("rw", lg)]
        t0 = time.perf_counter()
        y = oracle.fft(x)
        for g0 in range(0, b, 16):
            cs = abft.group_checksums(x[g0:g0 + 16], y[g0:g0 + 16], w=w, r=r)
            abft.verify_group(cs, n, min(16, b - g0), 2.0 ** -24, 4.0)
        tot_s += time.perf_counter() - t0
        tot_flops += flops(n, b)
        desc.append(f"2^{lg}x{b}")
    return tot_flops, tot_s, "per N of the sweep: " + ", ".join(desc)


def _oracle_worker(job):
    elems, seed, sweep = job
    return oracle_sample(elems, seed=seed, sweep=sweep)


class OraclePool:
    """The oracle on every host core: one spawned process per core, each
    timing its own bounded sample of the sweep (different seeds); a sample's
    time is the wall time of the whole pool."""

    THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                   "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")

    def __init__(self, workers: int):
        import multiprocessing as mp
        self.workers = workers
        # one thread per process: numpy's BLAS would otherwise start a thread
        # per core in every process (the children read these at start-up)
        saved = {k: os.environ.get(k) for k in self.THREAD_VARS}
        for k in self.THREAD_VARS:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(workers)
            self.pool.map(_oracle_worker, [(1 << 8, 0, [8])] * workers)     # start-up and imports
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def sample(self, elems_per_worker: int, seed0: int = 0, sweep=SWEEP):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(elems_per_worker, seed0 + 1000 * i, sweep)
                                             for i in range(self.workers)])
        wall = time.perf_counter() - t0
        return sum(r[0] for r in res), wall, f"{res[0][2]} on each of {self.workers} processes"

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    # every step: one N of the sweep in turn (2^18 elements, at least one
    # signal) on each host core; the steps cycle through the sweep, so K
    # steps weigh the N alike whatever K is, and each step stays under a few
    # seconds
    elems = 1 << 18
    cores = host_cores()
    pool = OraclePool(cores)
    for k in range(args.warmup):
        pool.sample(elems, sweep=[SWEEP[k % len(SWEEP)]])
    tf, ts, covered = 0.0, 0.0, []
    for k in range(args.steps):
        lg = SWEEP[k % len(SWEEP)]
        f, s, _ = pool.sample(elems, sweep=[lg])
        tf += f
        ts += s
        covered.append(lg)
    pool.close()
    desc = (f"one N per step in sweep order (log2 N: {sorted(set(covered))}), max(1, 2^18/N) signals "
            f"on each of {cores} processes")
    value = tf / ts / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ts / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched 1-D C2C FFT sweep N=2^8..2^24, batch*N=2^28, ABFT on "
                               "(bounded sample per step)", "sample": desc},
        "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import paper_2405_02520_gb300 as t
    from paper_2405_02520_gb300.inputs import uniform_batch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sweep = args.sweep

    total = 1 << args.total_log2
    x_host = uniform_batch(total, 1, seed=rank).reshape(-1)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    del x_host

    plans = {}
    for lg in sweep:
        n = 1 << lg
        plans[lg] = t.tfft_plan(n, total // n, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)

    def step(pl, timing_events=None):
        for lg in sweep:
            if timing_events is not None:
                timing_events[lg][0].record(stream)
            t.tfft_exec(pl[lg], x, y, stream)
            if timing_events is not None:
                timing_events[lg][1].record(stream)

    for _ in range(args.warmup):
        step(plans)
    torch.cuda.synchronize()
    for lg in sweep:
        t.tfft_reset_counters(plans[lg])
        t.tfft_set_timing(plans[lg], True)
        t.tfft_timing(plans[lg])          # drop warm-up records

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(local)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        s = str(uuid)
        gpu_id = s if s.startswith("GPU-") else "GPU-" + s
    sampler = ClockSampler(gpu_id)

    def new_events():
        return {lg: [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                     for _ in range(args.steps)] for lg in sweep}

    def timed_steps(pl, evs):
        for k in range(args.steps):
            step(pl, {lg: evs[lg][k] for lg in sweep})

    def per_n_total(evs):
        return {lg: sum(a.elapsed_time(b) for a, b in evs[lg]) / args.steps for lg in sweep}

    per_n = new_events()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    time.sleep(0.2)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    timed_steps(plans, per_n)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    max_ms = reduce_scalar(elapsed_ms, "max", dev)

    kinds = {k: [0.0, 0] for k in KERNEL_KINDS}
    launches = 0
    stats = {}
    for lg in sweep:
        tm = t.tfft_timing(plans[lg])
        for k, (ms, cnt) in tm.items():
            kinds[k][0] += ms
            kinds[k][1] += cnt
        st = t.tfft_report_ex(plans[lg])
        stats[lg] = st
        launches += st["launches"]
        t.tfft_set_timing(plans[lg], False)
    torch.cuda.synchronize()
    per_n_ms = per_n_total(per_n)

    flops_step = sum(flops(1 << lg, total >> lg) for lg in sweep)
    value = ws * args.steps * flops_step / (max_ms / 1e3) / 1e9

    # roofline of the dominant kernel: 16 B (8 read + 8 write) per element per pass
    bytes_per_launch = total * 16
    dom = max((k for k in KERNEL_KINDS if kinds[k][1] > 0), key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    peak, peak_src = measured_peaks()
    achieved = bytes_per_launch / (dom_ms / dom_n / 1e3) / 1e9
    passes = {lg: t.tfft_plan_info(plans[lg])["passes"] for lg in sweep}
    step_bytes = sum(passes[lg] * bytes_per_launch for lg in sweep)
    step_gbs = step_bytes * args.steps / (elapsed_ms / 1e3) / 1e9
    # the same with the fewest passes a plan needs (one tile up to 4096
    # points, two passes up to 2^26, Section IV-A): the bytes the method must
    # move, whatever decomposition this build picked
    min_bytes = sum(min_passes(1 << lg) * bytes_per_launch for lg in sweep)
    min_gbs = min_bytes * args.steps / (elapsed_ms / 1e3) / 1e9

    # ABFT off: same sweep, for the overhead
    for lg in sweep:
        t.tfft_destroy(plans[lg])
    off = {lg: t.tfft_plan(1 << lg, total >> lg, t.TFFT_C64, t.TFFT_ABFT_OFF) for lg in sweep}
    per_off = new_events()
    for _ in range(args.warmup):
        step(off)
    torch.cuda.synchronize()
    for lg in sweep:                      # the same per-launch instrumentation as the ABFT-on steps
        t.tfft_set_timing(off[lg], True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    timed_steps(off, per_off)
    e1.record(stream)
    torch.cuda.synchronize()
    off_ms = reduce_scalar(e0.elapsed_time(e1), "max", dev)
    off_per_n = per_n_total(per_off)
    for lg in sweep:
        t.tfft_set_timing(off[lg], False)
        t.tfft_destroy(off[lg])

    campaign = None if args.no_ragged else sweep_campaign(t, torch, x, y, stream, sweep, total)
    ragged = None if args.no_ragged else ragged_measure(t, torch, stream, args, peak)
    tensor = None if args.no_ragged else tc_measure(t, torch, stream, peak)
    ablation = None if args.no_ragged else one_sided_measure(t, torch, x, y, stream, args)
    small = None if args.no_ragged else config1_measure(t, torch, stream, peak)
    c128 = None if args.no_ragged else c128_measure(t, torch, stream, peak)

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        plans = {lg: t.tfft_plan(1 << lg, total >> lg, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
                 for lg in sweep}
        hin = torch.empty(total, dtype=torch.complex64, pin_memory=True)
        hin.copy_(x.cpu())
        hout = torch.empty(total, dtype=torch.complex64, pin_memory=True)
        del x, y
        torch.cuda.empty_cache()
        e2e_steps = max(1, min(args.steps, 3))
        e2e_ms = 0.0
        for rep in range(1 + e2e_steps):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for lg in sweep:
                t.tfft_exec_host(plans[lg], hin, hout, stream)
            dt = (time.perf_counter() - t0) * 1e3
            if rep > 0:
                e2e_ms += dt
        e2e_ms = reduce_scalar(e2e_ms, "max", dev)
        e2e = {"value": round(ws * e2e_steps * flops_step / (e2e_ms / 1e3) / 1e9, 2), "unit": "GFLOP/s",
               "h2d_bytes_per_step": len(sweep) * total * 8, "d2h_bytes_per_step": len(sweep) * total * 8,
               "steps": e2e_steps, "ms_per_step": round(e2e_ms / e2e_steps, 3)}
        for lg in sweep:
            t.tfft_destroy(plans[lg])

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        # all host cores (one spawned process per core), and one core
        cores = host_cores()
        pool = OraclePool(cores)
        f, s, desc = pool.sample(1 << 20)
        pool.close()
        one = OraclePool(1)
        f1, s1, desc1 = one.sample(1 << 22)
        one.close()
        cpu = {"value": round(f / s / 1e9, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": desc, "seconds": round(s, 2),
               "single_core": {"value": round(f1 / s1 / 1e9, 4), "sample": desc1, "seconds": round(s1, 2)}}

    if rank != 0:
        return 0
    clocks = sampler.summary()
    tr = recorded_traffic(dom, total)
    per_n_out = {}
    for lg in sweep:
        n = 1 << lg
        ms_on, ms_off = per_n_ms[lg], off_per_n[lg]
        per_n_out[str(lg)] = {
            "passes": passes[lg],
            "ms": round(ms_on, 4), "ms_abft_off": round(ms_off, 4),
            "gflops": round(flops(n, total // n) / (ms_on / 1e3) / 1e9, 1),
            "hbm_frac": round(passes[lg] * bytes_per_launch / (ms_on / 1e3) / 1e9 / peak, 4),
            "hbm_frac_min_passes": round(min_passes(n) * bytes_per_launch / (ms_on / 1e3) / 1e9 / peak, 4),
            "abft_overhead_pct": round((ms_on - ms_off) / ms_off * 100, 2),
            "max_clean_ratio": round(stats[lg]["max_clean_ratio"], 4),
        }
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(max_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"batched 1-D C2C FFT complex64, N=2^{sweep[0]}..2^{sweep[-1]} (one transform "
                        f"per N per step), batch*N=2^{args.total_log2} ({total * 8 / 2**30:g} GiB), "
                        "U[-1,1) re/im, two-sided ABFT on (G=16)",
            "sweep_log2n": sweep,
            "elements_per_transform": total,
            "parallelism": f"replicas x{ws} (weak scaling, no data-path collective)",
            "l2": f"inputs ({total * 8 / 2**30:g} GiB per transform) larger than L2",
        },
        "hbm_roofline_pct_step": round(100 * step_gbs / peak, 2),
        "hbm_roofline_pct_step_min_passes": round(100 * min_gbs / peak, 2),
        "abft_overhead_pct": round((max_ms - off_ms) / off_ms * 100, 2),
        "roofline": {
            "bound": "hbm",
            "kernel": dom,
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": tr,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "launches": dom_n,
        },
        "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in kinds.items() if v[1]},
        "per_n": per_n_out,
        "faults": {"detected": int(sum(s["detected"] for s in stats.values())),
                   "max_clean_ratio": max(s["max_clean_ratio"] for s in stats.values())},
        "sweep_campaign": campaign,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "ragged": ragged,
        "one_sided": ablation,
        "config1": small,
        "complex128": c128,
        "tensor_core": tensor,
    }
    print(json.dumps(line), flush=True)
    return 0


RAGGED_COUNT, RAGGED_LOG2 = 20000, (6, 16)


def ragged_measure(t, torch, stream, args, peak):
    """A ragged batch: 20,000 signals, log2 length uniform over {6..16},
    U[-1,1) re/im, seed 5, packed back to back; autotuned plan, graph-replayed
    execs, ABFT on and off, in the bucket-stream form (one plan per bucket on
    its own stream) and the persistent form (pass families: one persistent
    launch per pass role and sub-transform length pulling size-sorted items
    from an atomic counter); beside them the staged form (gather, transform,
    scatter) and one plan per length run one after another on the same
    signals grouped by length beforehand (the grouping not timed).  Bytes
    counted as algorithmic: 16 B per element per pass of each bucket's plan."""
    rng = np.random.default_rng(5)
    lengths = (1 << rng.integers(RAGGED_LOG2[0], RAGGED_LOG2[1] + 1, size=RAGGED_COUNT)).astype(np.int64)
    total = int(lengths.sum())
    xr = torch.empty(total, dtype=torch.complex64, device=stream.device)
    g = torch.Generator(device=stream.device).manual_seed(5)
    xr.real.uniform_(-1, 1, generator=g)
    xr.imag.uniform_(-1, 1, generator=g)
    yr = torch.empty_like(xr)
    out = {"signals": RAGGED_COUNT, "log2_lengths": list(RAGGED_LOG2), "elements": total, "seed": 5}
    for mode, key, staged, persistent in ((t.TFFT_ABFT_TWO_SIDED, "ms", False, False),
                                          (t.TFFT_ABFT_OFF, "ms_abft_off", False, False),
                                          (t.TFFT_ABFT_TWO_SIDED, "ms_persistent", False, True),
                                          (t.TFFT_ABFT_OFF, "ms_persistent_abft_off", False, True),
                                          (t.TFFT_ABFT_TWO_SIDED, "ms_staged", True, False)):
        r = t.Ragged(lengths.tolist(), abft_mode=mode, autotune=True, staged=staged, persistent=persistent)
        for _ in range(max(3, args.warmup)):
            r.exec(xr, yr, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(5, args.steps)
        e0.record(stream)
        for _ in range(k):
            r.exec(xr, yr, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[key] = round(e0.elapsed_time(e1) / k, 4)
        if key in ("ms", "ms_persistent"):
            info = dict(r.info())
            st = r.report()
            pre = "" if key == "ms" else "persistent_"
            out[pre + "detected_clean"] = st["detected"]
            if key == "ms":
                out["buckets"] = {str(n): p for n, p in sorted(info.items())}
                out["in_place_buckets"] = sum(r.layout().values())
            else:
                fams, pb = r.families()
                out["persistent_families"] = fams
                out["persistent_buckets"] = pb
            # one fault per 1000 signals, in distinct checksum groups, one exec
            sites = ragged_fault_sites(lengths, 1, seed=5)
            for k, i in enumerate(sites):
                n = int(lengths[i])
                r.set_fault(i, mode=t.TFFT_FAULT_SCALE, pass_=info[n] - 1, stage=0, line=0,
                            index=(7 * k + 1) % 16, factor=3.0)
            r.exec(xr, yr, stream)
            st2 = r.report()
            out[pre + "faults"] = {"injected": len(sites), "detected": st2["detected"] - st["detected"],
                                   "corrected": st2["corrected"] + st2["recomputed"] - st["corrected"]
                                   - st["recomputed"]}
        r.destroy()
    # one plan per length over the same signals grouped by length
    off = np.concatenate([[0], np.cumsum(lengths)])
    groups = []
    for n in sorted(set(lengths.tolist()), reverse=True):
        idx = np.nonzero(lengths == n)[0]
        sel = torch.from_numpy((off[idx][:, None] + np.arange(n)[None, :]).reshape(-1)).to(stream.device)
        xg = xr[sel].reshape(len(idx), n).contiguous()
        groups.append((t.tfft_plan(n, len(idx), t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED), xg, torch.empty_like(xg)))
        del sel
    for _ in range(max(3, args.warmup)):
        for pl, xg, yg in groups:
            t.tfft_exec(pl, xg, yg, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(5, args.steps)
    e0.record(stream)
    for _ in range(k):
        for pl, xg, yg in groups:
            t.tfft_exec(pl, xg, yg, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["ms_per_length_plans"] = round(e0.elapsed_time(e1) / k, 4)
    for pl, _, _ in groups:
        t.tfft_destroy(pl)
    del groups
    out["speedup_vs_per_length_plans"] = round(out["ms_per_length_plans"] / out["ms"], 3)
    fl = sum(float(flops(int(n), 1)) for n in lengths)
    passes = {int(n): p for n, p in ((int(k), v) for k, v in out["buckets"].items())}
    alg = sum(16.0 * passes[int(n)] * int(n) for n in lengths)
    out["gflops"] = round(fl / (out["ms"] / 1e3) / 1e9, 1)
    out["hbm_frac"] = round(alg / (out["ms"] / 1e3) / 1e9 / peak, 4)
    out["abft_overhead_pct"] = round((out["ms"] - out["ms_abft_off"]) / out["ms_abft_off"] * 100, 2)
    out["persistent_speedup_vs_bucket_streams"] = round(out["ms"] / out["ms_persistent"], 3)
    return out


def ragged_fault_sites(lengths, per_1000, seed):
    """Signals to fault: `per_1000` per 1000 signals, in distinct checksum
    groups (16 consecutive signals of one length), at most four per length
    (one below 256 points, where the armed sites after the first are not
    honoured)."""
    rng = np.random.default_rng(seed)
    want = max(1, len(lengths) * per_1000 // 1000)
    local, counts = {}, {}
    for i, n in enumerate(lengths):
        local[i] = counts.get(int(n), 0)
        counts[int(n)] = local[i] + 1
    used, per_len, out = set(), {}, []
    for i in rng.permutation(len(lengths)):
        n = int(lengths[i])
        g = (n, local[int(i)] // 16)
        if g in used or per_len.get(n, 0) >= (1 if n < 256 else 4):
            continue
        used.add(g)
        per_len[n] = per_len.get(n, 0) + 1
        out.append(int(i))
        if len(out) == want:
            break
    return out


def tc_measure(t, torch, stream, peak):
    """The radix-16 butterflies on FP32 CUDA cores and on the tensor cores
    (split TF32, split BF16, plain TF32) at N = 4096 x 65536 and 65536 x 4096 signals,
    N(0, 0.3^2) re/im, ABFT on.  Timing only; the error of each form against
    the oracle is measured by the tests."""
    out = {}
    for n, batch in ((4096, 65536), (65536, 4096)):
        xs = torch.empty((batch, n), dtype=torch.complex64, device=stream.device)
        g = torch.Generator(device=stream.device).manual_seed(4)
        xs.real.normal_(0, 0.3, generator=g)
        xs.imag.normal_(0, 0.3, generator=g)
        ys = torch.empty_like(xs)
        res = {}
        for name, prec in (("fp32", t.TFFT_PREC_FP32), ("tf32x3", t.TFFT_PREC_TF32X3),
                           ("bf16x3", t.TFFT_PREC_BF16X3), ("tf32", t.TFFT_PREC_TF32)):
            pl = t.tfft_plan_ex(n, batch, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, precision=prec)
            passes = t.tfft_plan_info(pl)["passes"]
            for _ in range(3):
                t.tfft_exec(pl, xs, ys, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                t.tfft_exec(pl, xs, ys, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            res[name] = {"ms": round(ms, 4), "gflops": round(flops(n, batch) / (ms / 1e3) / 1e9, 1),
                         "hbm_frac": round(16.0 * passes * n * batch / (ms / 1e3) / 1e9 / peak, 4),
                         "detected": t.tfft_report(pl)[0]}
            t.tfft_destroy(pl)
        out[f"{n}x{batch}"] = res
        del xs, ys
    return out


def config1_measure(t, torch, stream, peak):
    """N = 1024 x 256 signals, U[-1,1), ABFT on: 2 MiB in and out, so one pair
    of buffers stays in L2.  Timed hot (the same pair every exec) and over 64
    rotating pairs (128 MiB each way, more than L2) for the HBM figure."""
    n, b, pairs, k = 1024, 256, 64, 640
    xs = torch.empty((pairs, b, n), dtype=torch.complex64, device=stream.device)
    g = torch.Generator(device=stream.device).manual_seed(0)
    xs.real.uniform_(-1, 1, generator=g)
    xs.imag.uniform_(-1, 1, generator=g)
    ys = torch.empty_like(xs)
    pl = t.tfft_plan(n, b, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
    out = {"n": n, "batch": b}
    for name, rot in (("hot_l2", 1), ("rotating_64_pairs", pairs)):
        for i in range(8):
            t.tfft_exec(pl, xs[i % rot], ys[i % rot], stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(k):
            t.tfft_exec(pl, xs[i % rot], ys[i % rot], stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / k * 1e3
        out[name] = {"us_per_exec": round(us, 2), "gflops": round(flops(n, b) / (us / 1e6) / 1e9, 1),
                     "hbm_frac": round(16.0 * n * b / (us / 1e6) / 1e9 / peak, 4)}
    # the same exec captured once into a CUDA graph and replayed (this size
    # is launch-bound: the pass, the verification and the correction
    # launches that find nothing to do)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        t.tfft_exec(pl, xs[0], ys[0], torch.cuda.current_stream())
    for _ in range(8):
        g2.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k):
        g2.replay()
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / k * 1e3
    out["graph_replay_hot_l2"] = {"us_per_exec": round(us, 2), "gflops": round(flops(n, b) / (us / 1e6) / 1e9, 1)}
    out["detected"] = t.tfft_report(pl)[0]
    del g2
    t.tfft_destroy(pl)
    return out


# Real flops that the complex128 tile kernels execute per value, from their
# in-register DFTs (recursive radix 2 with the trivial roots free: DFT-2 4,
# DFT-4 16, DFT-8 56 and DFT-16 176 flops), their stage twiddles (one complex
# multiply, 6 flops, for E - 1 of every E values at each stage after the
# first) and the column passes' inter-pass twiddles (a complex multiply a
# value plus the recurrence that steps the twiddle along a thread's values).
# The checksum arithmetic is not counted.
C128_DFT_FLOPS = {1: 0, 2: 4, 4: 16, 8: 56, 16: 176}
C128_CMUL_FLOPS = 6.0


def sweep_campaign(t, torch, x, y, stream, sweep, total, launches=100):
    """The complex64 sweep at its full size (2^28 elements per N) with one
    random bit flip per `launches` launches: at each N, a random launch of
    `launches` carries one flip at a random (pass, stage, signal, line,
    element, bit).  The fault is classified on a detect-only plan (harmful:
    the faulty signal's output misses 2e-6 log2 N relative L2), and after the
    corrected launch every signal is compared with the clean output of the
    same plan (the library's own output, which the parity tests hold to the
    oracle; the 2 GiB batch is too large for the oracle here).  Clean
    launches count as false-positive opportunities."""
    import numpy as np
    out = {"launches": 0, "injected": 0, "harmful": 0, "harmful_detected": 0, "harmful_located": 0,
           "harmful_corrected": 0, "benign": 0, "benign_output_ok": 0, "false_positives": 0, "sites": []}
    ref = torch.empty_like(y)
    for lg in sweep:
        n = 1 << lg
        b = total // n
        tol = 2e-6 * lg
        rng = np.random.default_rng(2000 + lg)
        pl = t.tfft_plan(n, b, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED)
        det = t.tfft_plan_ex(n, b, t.TFFT_C64, t.TFFT_ABFT_TWO_SIDED, detect_only=True)
        info = t.tfft_plan_info(pl)
        p = int(rng.integers(info["passes"]))
        site = dict(mode=t.TFFT_FAULT_BITFLIP, pass_=p, stage=int(rng.integers(-1, info["stages"][p])),
                    signal=int(rng.integers(b)), line=int(rng.integers(info["lines_per_signal"][p])),
                    index=int(rng.integers(info["nsub"][p])), bit=int(rng.integers(64)), factor=0.0)
        at = int(rng.integers(launches))
        t.tfft_exec(pl, x, ref, stream)
        ref_norm = torch.linalg.vector_norm(ref.view(b, n), dim=1)

        def row_err():
            with torch.no_grad():
                e = torch.linalg.vector_norm((y - ref).view(b, n), dim=1) / ref_norm
            return torch.nan_to_num(e, nan=float("inf")).cpu().numpy()

        t.tfft_set_fault(det, **site)
        t.tfft_exec(det, x, y, stream)
        harmful = bool(row_err()[site["signal"]] > tol)
        t.tfft_reset_counters(pl)
        for k in range(launches):
            before = t.tfft_report(pl)[0] if k == at else None
            if k == at:
                t.tfft_set_fault(pl, **site)
            t.tfft_exec(pl, x, y, stream)
            if k == at:
                d = t.tfft_report(pl)[0] > before
                ev, _ = t.tfft_fault_log(pl, 1)
                loc = d and ev and ev[-1]["signal"] == site["signal"]
                ok = bool(np.all(row_err() <= tol))
        st = t.tfft_report_ex(pl)
        out["launches"] += launches
        out["injected"] += 1
        out["false_positives"] += int(st["detected"]) - int(d)
        if harmful:
            out["harmful"] += 1
            out["harmful_detected"] += int(d)
            out["harmful_located"] += int(bool(loc))
            out["harmful_corrected"] += int(ok)
        else:
            out["benign"] += 1
            out["benign_output_ok"] += int(ok)
        out["sites"].append(dict(log2n=lg, launch=at, harmful=harmful, detected=bool(d), **{
            k: v for k, v in site.items() if k not in ("mode", "factor")}))
        t.tfft_destroy(pl)
        t.tfft_destroy(det)
    del ref
    return out


def c128_executed_flops(n, b, info):
    """Flops the complex128 passes of a plan execute on their FFT arithmetic:
    a pass of S stages over nsub values is a radix-R0 stage then S - 1 of
    radix E (16 where S is log2(nsub) / 4 rounded up and differs from the
    radix-8 count, else 8), R0 = nsub / E^(S-1)."""
    import math
    per = 0.0
    for i in range(info["passes"]):
        nsub, st = info["nsub"][i], info["stages"][i]
        lg = int(round(math.log2(nsub)))
        e = 16 if st == -(-lg // 4) and st != -(-lg // 3) else 8
        r0 = nsub // e ** (st - 1)
        per += C128_DFT_FLOPS[r0] / r0 + (st - 1) * (C128_DFT_FLOPS[e] / e + C128_CMUL_FLOPS * (e - 1) / e)
        if i < info["passes"] - 1:          # inter-pass twiddle of this column pass
            per += C128_CMUL_FLOPS * (1 + (e - 1) / e)
    return b * n * per


def c128_measure(t, torch, stream, peak):
    """complex128, N(0,1) re/im: N = 2^20 x 64 and N = 2^12 x 2^14, ABFT on
    and off.  Bytes: 32 B per element per pass.  The FP64 units bound these
    transforms on this part, so the line also gives the FP64 fraction: the
    flops the radix-8 kernels execute (c128_executed_flops) over the FP64
    multiply-add peak measured here (tfft_measure_fma_peak)."""
    fp64 = t.tfft_measure_fma_peak(True, 4000)
    out = {"fp64_peak_measured_tflops": round(fp64, 3), "fp64_nominal_tflops": 1.25,
           "executed_flops": "in-register DFTs (DFT-8 56, DFT-16 176 flops), stage twiddles "
                             "(6 flops for (E-1)/E of the values at each later stage), inter-pass "
                             "twiddles and their recurrence; checksums not counted"}
    for lg, b in ((20, 64), (12, 1 << 14)):
        n = 1 << lg
        xs = torch.empty((b, n), dtype=torch.complex128, device=stream.device)
        g = torch.Generator(device=stream.device).manual_seed(3)
        xs.real.normal_(0, 1, generator=g)
        xs.imag.normal_(0, 1, generator=g)
        ys = torch.empty_like(xs)
        res = {}
        for name, mode in (("on", t.TFFT_ABFT_TWO_SIDED), ("off", t.TFFT_ABFT_OFF)):
            pl = t.tfft_plan(n, b, t.TFFT_C128, mode)
            info = t.tfft_plan_info(pl)
            passes = info["passes"]
            for _ in range(3):
                t.tfft_exec(pl, xs, ys, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                t.tfft_exec(pl, xs, ys, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            res[f"ms_{name}"] = round(ms, 4)
            if name == "on":
                res["passes"] = passes
                res["gflops"] = round(flops(n, b) / (ms / 1e3) / 1e9, 1)
                res["hbm_frac"] = round(32.0 * passes * n * b / (ms / 1e3) / 1e9 / peak, 4)
                ex = c128_executed_flops(n, b, info)
                res["executed_tflops"] = round(ex / (ms / 1e3) / 1e12, 4)
                res["fp64_frac"] = round(ex / (ms / 1e3) / 1e12 / fp64, 4)
                res["detected"] = t.tfft_report(pl)[0]
            t.tfft_destroy(pl)
        res["abft_overhead_pct"] = round((res["ms_on"] - res["ms_off"]) / res["ms_off"] * 100, 2)
        out[f"{n}x{b}"] = res
        del xs, ys
    return out


def one_sided_measure(t, torch, x, y, stream, args):
    """The one-sided ABFT mode (per-signal checks, recompute on detection) as
    an ablation of the two-sided scheme: N = 2^10 and 2^16, 2^28 elements."""
    out = {}
    total = x.numel()
    for lg in (10, 16):
        n = 1 << lg
        ms = {}
        for name, mode in (("two_sided", t.TFFT_ABFT_TWO_SIDED), ("one_sided", t.TFFT_ABFT_ONE_SIDED),
                           ("off", t.TFFT_ABFT_OFF)):
            pl = t.tfft_plan(n, total // n, t.TFFT_C64, mode)
            for _ in range(3):
                t.tfft_exec(pl, x, y, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                t.tfft_exec(pl, x, y, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[name] = e0.elapsed_time(e1) / 5
            t.tfft_destroy(pl)
        out[str(lg)] = {k: round(v, 4) for k, v in ms.items()}
        out[str(lg)]["overhead_pct"] = {k: round((ms[k] - ms["off"]) / ms["off"] * 100, 2)
                                        for k in ("two_sided", "one_sided")}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--sweep", type=lambda s: [int(v) for v in s.split(",")], default=SWEEP,
                    help="comma-separated log2 N values (default 8..24)")
    ap.add_argument("--total-log2", type=int, default=TOTAL_LOG2,
                    help="log2 of the elements per transform (default 28; smaller for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the ragged-batch, one-sided-mode and tensor-core measurements")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)      # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
