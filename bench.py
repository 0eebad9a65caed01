#!/usr/bin/env python3
"""Benchmark: Pauli terms/s of the exact XOR-FWHT M2 at N = 20 on GB300.

One step = one full M2 evaluation of an N = 20 Haar-random state (complex64;
by default the FP16 hi/lo split mode, whose Hadamard stages run on the
tensor cores, --mode fp32 for the CUDA-core path): all 4^20 = 1.1e12 Pauli
strings X^x Z^z, i.e. every row of the hot path (norm, XOR-shifted
products, FWHT, |A|^4 reduction, FP64 sum, log2), |dM2| against the FP64
oracle's value of the same state reported beside it.
The state is resident in HBM before the timed region; the L2 is flushed
(a 512 MiB write) between timed steps, outside the per-step CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 is launched with torchrun: every rank evaluates its own state (weak
scaling, no data-path collective; the barrier and the max over ranks are
timing only).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload on the host cores (rank 0 only).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Pauli terms/s at N=20 within |dM2|<=1e-6 vs FP64; serve p50/p99 latency"
UNIT = "Pauli terms/s"
N_QUBITS = 20
CONFIG_INDEX = 2  # seeds: 1000 * config + state


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--N", type=int, default=N_QUBITS)
    ap.add_argument("--mode", default="fp16_split",
                    help="fp16_split (tensor cores, the fastest within the tolerance), bf16_split, fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="all",
                    help="comma list of extras to run: serving, batched, batched_fp16_split, fp64_check, "
                         "modes, orders, brickwork_dynamics, tfim_quench (default all)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="seconds of Poisson arrivals per load point (300 for the 5-minute trace)")
    ap.add_argument("--serve-fifo-seconds", type=float, default=None,
                    help="replay only this many seconds of each trace in the one-launch-per-request arm")
    ap.add_argument("--serve-loads", default="0.25,0.5,0.75",
                    help="load points, as fractions of the capacity measured at N = 20")
    ap.add_argument("--batch-states", type=int, default=512)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        pw = [num(r[3]) for r in self.rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


# --------------------------------------------------------------- oracle arm

def cpu_oracle_sample(N: int, seconds: float, seed: int):
    """Time the FP64 oracle (Algorithm 1, OpenMP over shifts) on a bounded
    sample of shifts of the same N=20 state.  Returns (terms/s, cores, sample)."""
    import numpy as np

    import oracle
    from paper_2512_24685_gb300 import workloads as W
    psi = W.haar_state(N, seed, np.complex64)
    cores = oracle.num_threads()
    d = 1 << N
    n = max(1, cores)  # calibration: one shift per thread
    t0 = time.perf_counter()
    oracle.sum4_xorfwht(psi, 0, n)
    dt = time.perf_counter() - t0
    n_big = int(max(cores, min(d, n * max(1.0, seconds / max(dt, 1e-6)))))
    n_big = max(cores, (n_big // cores) * cores)
    t0 = time.perf_counter()
    oracle.sum4_xorfwht(psi, n, n + n_big)
    dt = time.perf_counter() - t0
    return n_big * d / dt, cores, f"N={N} Haar state (complex64 widened to FP64), shifts [{n}, {n + n_big}) of {d}: {n_big * d:.3e} Pauli terms in {dt:.1f} s"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    N = args.N
    d = 1 << N
    per_step_s = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    import numpy as np
    from paper_2512_24685_gb300 import workloads as W
    psi = W.haar_state(N, W.config_seed(CONFIG_INDEX, 0), np.complex64)
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    oracle.sum4_xorfwht(psi, 0, cores)
    cal = (time.perf_counter() - t0) / cores  # seconds per shift (parallel)
    n_step = max(cores, int(per_step_s / max(cal, 1e-9)) // cores * cores)
    x = cores
    times = []
    for k in range(args.warmup + args.steps):
        a = x % d
        b = min(d, a + n_step)
        t0 = time.perf_counter()
        oracle.sum4_xorfwht(psi, a, b)
        dt = time.perf_counter() - t0
        x = b
        if k >= args.warmup:
            times.append((b - a) * d / dt)
    value = statistics.mean(times)
    total = sum(n_step * d / v for v in times)
    sample = f"each step: {n_step} shifts of the N={N} Haar state ({n_step * d:.3e} Pauli terms), FP64 oracle, {cores} threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"N={N} Haar-random state (complex64), all 4^{N} Pauli strings per step",
                   "N": N, "states_per_gpu": 1, "parallelism": f"replicas x{args.gpus}",
                   "sample": "each step evaluates a bounded range of shifts (see cpu_baseline.sample); "
                             "the throughput is Pauli terms of that range per second"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0



# ------------------------------------------------------------------ extras

def _serving_pool(torch, W, n_lo=10, n_hi=20):
    """One state per family (Haar, product, stabilizer, depth-8 brickwork) per
    N, complex64, on the device."""
    import numpy as np
    pool = {}
    for n in range(n_lo, n_hi + 1):
        seed = W.config_seed(4, 10 * n)
        pool[(n, 0)] = torch.from_numpy(W.haar_state(n, seed, np.complex64)).cuda()
        pool[(n, 1)] = torch.from_numpy(W.product_state(n, seed + 1, np.complex64)[0]).cuda()
        pool[(n, 2)] = W.stabilizer_state_torch(n, seed + 2, "cuda", dtype=torch.complex64).contiguous()
        pool[(n, 3)] = W.brickwork_state_torch(n, 8, seed + 3, "cuda", dtype=torch.complex64).contiguous()
    torch.cuda.synchronize()
    return pool


def _serving_trace(rate, seconds, seed, W):
    import numpy as np
    rng = W.rng_for(seed)
    ns, p = W.serving_n_distribution()
    t, trace = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        trace.append((t, int(rng.choice(ns, p=p)), int(rng.integers(4))))
    return trace


def _pct(lat, q):
    return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))] if lat else None


def run_serving(binding, torch, W, terms_per_s, seconds, loads, mode, chunk_terms=1 << 37, fifo_seconds=None):
    """Poisson arrivals at each of `loads` x measured capacity: through the
    server (slots with the autotuned two-pass plans of N = 17..20, large
    requests split into shift ranges of <= chunk_terms Pauli terms that take
    turns with the rest), and the same trace with one synchronous launch per
    request in arrival order (FIFO) on plans created and tuned before its
    clock starts (on the first fifo_seconds of each trace, default all of
    it).  Both arms use the arithmetic mode `mode`."""
    import threading as th
    ns, p = W.serving_n_distribution()
    mean_work = float(sum(pn * 4.0 ** n for n, pn in zip(ns, p)))
    capacity = terms_per_s / mean_work
    pool = _serving_pool(torch, W)
    tunings = {}
    for n in range(17, 21):
        with binding.Plan(n, "c64", mode) as pl:
            tunings[n], _ = pl.autotune(n)
    # the FIFO arm's plans, tuned the same way, exist before any clock starts
    plans = {}
    for n in range(min(ns), max(ns) + 1):
        plans[n] = binding.Plan(n, "c64", mode)
        if n in tunings:
            plans[n].set_tuning(**tunings[n])
        plans[n].m2(pool[(n, 0)])  # warm-up
    torch.cuda.synchronize()
    out = {"capacity_per_s": capacity, "seconds_per_load": seconds, "mean_terms_per_request": mean_work,
           "mode": mode, "chunk_terms": chunk_terms,
           "n_mix": "P(N) ~ 2^-(N-10)/2, N in 10..20; Haar/product/stabilizer/brickwork", "loads": {}}
    for li, load in enumerate(loads):
        rate = load * capacity
        trace = _serving_trace(rate, seconds, 4242 + li, W)
        res = {"arrival_rate_per_s": rate, "requests": len(trace)}
        with binding.Server(max_inflight=4, max_N=20, hbm_budget_bytes=16 << 30, mode=mode,
                            slot_scratch_bytes=192 << 20, chunk_terms=chunk_terms) as srv:
            for n, t in tunings.items():
                srv.set_tuning(n, t)
            t0 = time.perf_counter()
            tickets = []
            for (ta, n, fam) in trace:
                dt = t0 + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(srv.submit(pool[(n, fam)]))
            for tk in tickets:
                srv.wait(tk, 600000)
            st = srv.stats()
        res["server"] = {k: st[k] for k in ("p50_latency_ms", "p99_latency_ms", "mean_latency_ms",
                                            "states_per_s", "pauli_terms_per_s", "completed", "failed",
                                            "rejected", "peak_resident_bytes")}
        # one launch per request, FIFO, same arrivals
        if fifo_seconds is not None:
            trace = [r for r in trace if r[0] <= fifo_seconds]
            res["fifo_seconds"] = fifo_seconds
        lat = []
        q, lock, done_ev = [], th.Lock(), th.Event()

        def worker():
            idx = 0
            while idx < len(trace):
                with lock:
                    ready = idx < len(q)
                if not ready:
                    time.sleep(0.0002)
                    continue
                (ta_abs, n, fam) = q[idx]
                plans[n].m2(pool[(n, fam)])
                lat.append((time.perf_counter() - ta_abs) * 1000.0)
                idx += 1
            done_ev.set()

        w = th.Thread(target=worker)
        w.start()
        t0 = time.perf_counter()
        for (ta, n, fam) in trace:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            with lock:
                q.append((time.perf_counter(), n, fam))
        done_ev.wait()
        w.join()
        span = max(1e-9, time.perf_counter() - t0)
        lat.sort()
        res["one_launch_per_request"] = {"p50_latency_ms": _pct(lat, 0.50), "p99_latency_ms": _pct(lat, 0.99),
                                         "mean_latency_ms": sum(lat) / len(lat) if lat else None,
                                         "states_per_s": len(lat) / span}
        out["loads"][f"{load:g}"] = res
    for pl in plans.values():
        pl.close()
    return out


def run_batched(binding, torch, W, count, mode="fp32"):
    """The uneven batched workload: `count` brickwork states, N ~ U{12..18},
    depth ~ U{1..32}, one sre_m2_batched submission replayed from its graph,
    in arithmetic mode `mode` (split modes: the N = 16..18 classes on the
    tensor cores)."""
    spec = W.uneven_batch_spec(count=count)
    states = [W.brickwork_state_torch(n, t, s, "cuda", dtype=torch.complex64).contiguous()
              for n, t, s in spec]
    terms = float(sum(4.0 ** n for n, _, _ in spec))
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with binding.Plan(18, "c64", mode) as plan, torch.cuda.stream(side):
        for n in ((18, 17, 16) if mode != "fp32" else (18, 17)):
            plan.autotune(n)
        out = torch.empty(count, dtype=torch.float64, device="cuda")
        plan.m2_batched(states, out=out)  # eager run + graph capture
        plan.m2_batched(states, out=out)  # first replay
        side.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = plan.launch_count()
        e0.record(side)
        plan.m2_batched(states, out=out)
        e1.record(side)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        launches = plan.launch_count() - l0
    return {"states": count, "pauli_terms": terms, "ms": ms, "states_per_s": count / (ms / 1e3),
            "pauli_terms_per_s": terms / (ms / 1e3), "gpu_launches": launches,
            "mode": mode,
            "workload": "brickwork Haar circuits on |0^N>, N ~ U{12..18}, depth ~ U{1..32}, complex64"}


def golden_m2(N, dtype_name):
    """The FP64 oracle's M2 of the benchmark state (tests/golden, written by
    the oracle-only script make_n20_oracle.py), or None."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "n20_haar_oracle.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(dtype_name)
    except (OSError, ValueError):
        return None
    return rec["m2"] if rec and rec.get("N") == N else None


def tc_mma_flops(N):
    """Executed MMA flops of the tensor-core kernel for one evaluation: each
    halved shift (x >= 4096) has 2^(N-13) tiles of 8192 real values per pass,
    and every tile is one stage of eight M = 128, N = 128, K = 16 MMAs."""
    if N < 16 or N > 20:
        return 0.0
    tiles = 2.0 ** (N - 13) * 2  # both passes
    return ((1 << N) - 4096) * tiles * 8 * (2.0 * 128 * 128 * 16)


def run_modes(binding, torch, W, N, head_mode, head, peaks):
    """Every FP32-input arithmetic mode on the benchmark's N = 20 state,
    side by side: autotuned plan, 3 timed evaluations after a warm-up,
    the main launch's CUDA-event time (sre_plan_last_kernel_ms), |dM2|
    against the oracle's golden value, and the roofline of that launch
    (FP32: algorithmic ops over the FP32 lanes; split modes: executed MMA
    flops over the measured bf16 peak).  The headline mode's own figures
    (`head`) are reused instead of measured again."""
    import numpy as np
    psi = torch.from_numpy(W.haar_state(N, W.config_seed(CONFIG_INDEX, 0), np.complex64)).cuda()
    d = 1 << N
    ref = golden_m2(N, "complex64")
    sms = torch.cuda.get_device_properties(psi.device).multi_processor_count
    alu_peak = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    peak_s = peaks.get("bf16_tflops_sustained", 1700.0)
    peak_b = peaks.get("bf16_tflops", 1900.0)
    out = {}
    for mode in ("fp32", "fp16_split", "bf16_split"):
        if mode == head_mode:
            r = dict(head)
        else:
            with binding.Plan(N, "c64", mode) as p:
                tuning, _ = p.autotune(N)
                p.set_profiling(True)
                p.m2(psi)
                torch.cuda.synchronize()
                kms, walls = [], []
                for _ in range(3):
                    t0 = time.perf_counter()
                    m = p.m2(psi)
                    walls.append(time.perf_counter() - t0)
                    kms.append(p.last_kernel_ms()[0])
                kname = p.last_kernel_ms()[1]
            r = {"ms": statistics.mean(walls) * 1e3, "kernel_ms": statistics.mean(kms), "kernel": kname,
                 "m2": m, "tuning": tuning}
        kms_m = r["kernel_ms"]
        r["pauli_terms_per_s"] = float(d) * d / (r["ms"] * 1e-3)
        r["abs_diff_vs_oracle"] = abs(r["m2"] - ref) if ref is not None else None
        if mode == "fp32":
            r["alu_roofline_frac"] = (2 * N + 11) * float(d) * (d - 4096) / (kms_m * 1e-3) / alu_peak
        else:
            flops = tc_mma_flops(N)
            r["mma_flops_executed"] = flops
            r["mma_tflops_executed"] = flops / (kms_m * 1e-3) / 1e12
            r["tensor_roofline_frac"] = flops / (kms_m * 1e-3) / (peak_s * 1e12)
            r["tensor_roofline_frac_vs_burst"] = flops / (kms_m * 1e-3) / (peak_b * 1e12)
        out[mode] = r
    for mode in ("fp16_split", "bf16_split"):
        out[mode]["vs_fp32_time"] = out[mode]["ms"] / out["fp32"]["ms"]
        out[mode]["vs_fp32_kernel_time"] = out[mode]["kernel_ms"] / out["fp32"]["kernel_ms"]
    out["note"] = ("split modes: both passes' Hadamard stages as tcgen05 MMAs (pass 1: 4 register bits, one "
                   "H_128 stage, one accumulator butterfly; pass 2: one H_128 or I x H_{2^h2} stage) on "
                   "fixed-point hi/lo pieces, FP32 accumulate in TMEM; kernel_ms is the launch of the halved "
                   "shifts x >= 4096 alone; tensor peak = measured bf16 sustained (burst alongside)")
    return out


def run_fp64_check(binding, torch, W, N=20):
    """The FP64 path on the complex128 benchmark state at N = 20: one
    evaluation's time and |dM2| against the oracle's golden value."""
    import numpy as np
    psi = W.haar_state(N, W.config_seed(CONFIG_INDEX, 0), np.complex128)
    t = torch.from_numpy(psi).cuda()
    ref = golden_m2(N, "complex128")
    with binding.Plan(N, "c128", "fp64") as p:
        p.set_profiling(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = p.m2(t)
        ms = (time.perf_counter() - t0) * 1e3
        kms, kname = p.last_kernel_ms()
    return {"N": N, "dtype": "complex128", "mode": "fp64", "ms": ms, "kernel_ms": kms, "kernel": kname,
            "m2": m, "abs_diff_vs_oracle": abs(m - ref) if ref is not None else None,
            "pauli_terms_per_s": float(1 << N) ** 2 / (ms * 1e-3),
            "note": "one evaluation, no warm-up (default FP64 tuning); tolerance 1e-10"}


def run_orders(binding, torch, W, N, fp32_ms, m2_val, orders=(3, 4)):
    """Higher Renyi orders (Eq. (sre)) on the benchmark's N = 20 state: one
    timed sre_m_alpha per order (after a warm-up), beside the M2 time, with
    the tuning the autotuner picked for M2."""
    import numpy as np
    psi = torch.from_numpy(W.haar_state(N, W.config_seed(CONFIG_INDEX, 0), np.complex64)).cuda()
    out = {"N": N, "m2_kernel_ms": fp32_ms, "m2": m2_val}
    with binding.Plan(N, "c64") as p:
        p.autotune(N)
        for a in orders:
            p.m_alpha(psi, a)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m = p.m_alpha(psi, a)
            ms = (time.perf_counter() - t0) * 1e3
            out[f"alpha{a}"] = {"ms": ms, "m_alpha": m, "pauli_terms_per_s": 4.0 ** N / (ms / 1e3)}
    return out


def run_brickwork(binding, torch, W, cases=((14, 100, 20), (16, 100, 4))):
    """Example 2's dynamics on the device: S realizations of N-qubit Haar
    brickwork circuits from |0...0>, T steps, M2 of every realization after
    every step (sre_brickwork_m2_series, FP32 M2 of complex128 states)."""
    import math
    out = {}
    for N, S, T in cases:
        gates = torch.from_numpy(W.brickwork_gate_tensor(N, S, T)).cuda()
        with binding.Plan(N, "c128", "fp32") as p:
            p.brickwork_m2_series(gates[:1])  # warm-up (first-step graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2, _ = p.brickwork_m2_series(gates)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
        last = m2[-1].double()
        out[f"N{N}"] = {"realizations": S, "steps": T, "ms": ms, "ms_per_step": ms / T,
                        "pauli_terms_per_s": S * T * 4.0 ** N / (ms / 1e3),
                        "m2_last_step_mean": float(last.mean()), "m2_first_step_mean": float(m2[0].double().mean()),
                        "haar_value": math.log2(2 ** N + 3) - 2}
    return out


def run_tfim(binding, torch, W, cases=((14, 100, 10), (16, 100, 3)), dt=0.2):
    """Example 1's quench on the device: S random product states of N qubits
    evolved by the TFIM with longitudinal field (J = 1, hx = hz = 1.5), T steps
    of dt, M2 of every state after every step (sre_tfim_m2_series, FP32 M2 of
    complex128 states)."""
    import math
    import numpy as np
    out = {}
    for N, S, T in cases:
        psi0 = np.stack([W.product_state(N, W.config_seed(5, s))[0] for s in range(S)])
        with binding.Plan(N, "c128", "fp32") as p:
            warm = torch.from_numpy(psi0.copy()).cuda()
            p.tfim_m2_series(warm, 1, dt)  # warm-up (first-step graph capture)
            states = torch.from_numpy(psi0.copy()).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = p.tfim_m2_series(states, T, dt)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
        out[f"N{N}"] = {"realizations": S, "steps": T, "dt": dt, "ms": ms, "ms_per_step": ms / T,
                        "pauli_terms_per_s": S * T * 4.0 ** N / (ms / 1e3),
                        "m2_first_step_mean": float(m2[0].double().mean()),
                        "m2_last_step_mean": float(m2[-1].double().mean()),
                        "haar_value": math.log2(2 ** N + 3) - 2}
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the halved
# launch, from one ncu capture of a 16384-shift slice at N = 20 per mode and
# tuning, scaled by shifts to the 2^20 - 4096 halved shifts of one
# evaluation.  Valid only for that kernel build and tuning; any other run
# reports null.
TRAFFIC = {
    # FP32 CUDA-core two-pass kernel, its autotuned tuning (read + written on the slice)
    ("fp32", (0, 47, 23, 3, 3)): 45.449725e9 + 61.593259e9,
    # tensor-core kernel, FP16 pieces, the tunings its autotuner picks
    # (read + written on the slice)
    ("fp16_split", (3, 6, 2, 4, 0)): 45.709644e9 + 59.002857e9,
    ("fp16_split", (3, 6, 2, 5, 0)): 69.958212e9 + 68.431478e9,
    ("fp16_split", (2, 12, 3, 5, 1)): 54.314441e9 + 66.705181e9,
}
TRAFFIC_SLICE_SHIFTS = 16384
TRAFFIC_SOURCE = ("ncu --set full, 16384 halved shifts at N=20, scaled by shifts "
                  "to the halved launch (the x < 4096 launch adds < 1 %)")


def profiled_traffic(N, mode, tuning):
    if N != 20 or not tuning:
        return None
    key = (mode, (tuning["x_batch_log"], tuning["ring_slots"], tuning["lag"], tuning["pass2_tiles_log"],
                  tuning["pass1_blocks_log"]))
    b = TRAFFIC.get(key)
    if b is None:
        return None
    return b * ((1 << N) - 4096) / TRAFFIC_SLICE_SHIFTS


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2512_24685_gb300 import binding, workloads as W
    binding.load_library()
    N = args.N
    d = 1 << N
    terms = float(d) * float(d)
    psi_np = W.haar_state(N, W.config_seed(CONFIG_INDEX, rank), np.complex64)
    psi = torch.from_numpy(psi_np).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    plan = binding.Plan(N, "c64", args.mode)
    tuning, tune_ms = None, None
    if N > 12 and not args.no_autotune:
        tuning, tune_ms = plan.autotune(N)
    elif N > 12:
        tuning = plan.get_tuning(N)
    plan.set_profiling(True)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        plan.m2(psi)
    barrier()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)

    launches0 = plan.launch_count()
    step_ms, kern_ms = [], []
    barrier()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.m2_async(psi, out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(plan.last_kernel_ms()[0])
    barrier()
    wall = time.perf_counter() - wall0
    launches = plan.launch_count() - launches0
    kname = plan.last_kernel_ms()[1]
    m2_val = out.item()
    if sampler:
        time.sleep(0.2)
        sampler.stop()

    elapsed_s = sum(step_ms) / 1000.0
    if dist is not None:
        t = torch.tensor([elapsed_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = t.item()
    value = world * args.steps * terms / elapsed_s

    # ---- end to end through the public host entry point (pinned host buffer)
    e2e = None
    if not args.no_e2e:
        psi_h = torch.from_numpy(psi_np).pin_memory()
        plan.m2_host(psi_h)
        barrier()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.m2_host(psi_h)
            e2e_s += time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = t.item()
        launches += 0
        e2e = {"value": world * args.steps * terms / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(psi_h.numel() * psi_h.element_size()),
               "d2h_bytes_per_step": 32}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    clocks = sampler.summary() if sampler else {}
    max_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # FP32 ALU roofline: SMs x 128 FP32 lanes x max SM clock (one add / mul /
    # fma per lane per clock); algorithmic ops (2N + 11) d per Pauli term,
    # over the terms of the timed launch (the halved shifts x >= 4096; the
    # plan's profiling events bracket that launch alone)
    timed_terms = float(d) * (d - 4096) if N > 12 else terms
    alg_ops = (2 * N + 11) * timed_terms
    kern_s = statistics.mean(kern_ms) / 1000.0
    if args.mode == "fp64":
        peak_ops = None
    else:
        peak_ops = sms * 128 * max_mhz * 1e6
    achieved = alg_ops / kern_s
    roof = {
        "bound": "alu", "kernel": kname,
        "achieved": achieved / 1e12, "peak": (peak_ops / 1e12) if peak_ops else None,
        "unit": "TFLOP/s", "frac": (achieved / peak_ops) if peak_ops else None,
        "traffic": profiled_traffic(N, args.mode, tuning),
        "traffic_source": TRAFFIC_SOURCE,
        "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz (sm max); clocks {peak_src}",
        "alg_ops_per_launch": alg_ops, "kernel_ms": statistics.mean(kern_ms),
    }
    if clocks.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (sms * 128 * clocks["sm_mhz"] * 1e6)
    if args.mode in ("bf16_split", "fp16_split") and tc_mma_flops(N) > 0:
        # tensor-core modes: the dominant kernel is bound by the tensor pipe
        tflops = tc_mma_flops(N) / kern_s / 1e12
        peak_t = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {
            "bound": "tensor", "kernel": kname, "achieved": tflops, "peak": peak_t, "unit": "TFLOP/s",
            "frac": tflops / peak_t, "traffic": profiled_traffic(N, args.mode, tuning),
            "traffic_source": TRAFFIC_SOURCE,
            "peak_source": f"MEASURED_PEAKS bf16_tflops_sustained ({peak_src}); fp16 runs at the bf16 rate",
            "mma_flops_per_launch": tc_mma_flops(N), "kernel_ms": statistics.mean(kern_ms),
            "alu_frac_algorithmic": achieved / peak_ops if peak_ops else None,
        }

    cpu = None
    if not args.no_cpu_baseline and world >= 1:
        v, cores, sample = cpu_oracle_sample(N, args.cpu_seconds, W.config_seed(CONFIG_INDEX, 0))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    peaks, peak_src = load_peaks()
    extras = {}
    want = set(args.extras.split(",")) if not args.no_extras else set()

    def extra(name, fn):
        if name in want or "all" in want:
            try:
                extras[name] = fn()
            except Exception as exc:  # reported, not hidden
                extras[name] = {"error": repr(exc)}

    head = {"ms": statistics.mean(step_ms), "kernel_ms": statistics.mean(kern_ms), "kernel": kname,
            "m2": m2_val, "tuning": tuning}
    extra("serving", lambda: run_serving(binding, torch, W, value / world, args.serve_seconds,
                                         [float(v) for v in args.serve_loads.split(",")], args.mode,
                                         fifo_seconds=args.serve_fifo_seconds))
    extra("batched", lambda: run_batched(binding, torch, W, args.batch_states, "fp32"))
    extra("batched_fp16_split", lambda: run_batched(binding, torch, W, args.batch_states, "fp16_split"))
    extra("fp64_check", lambda: run_fp64_check(binding, torch, W))
    extra("modes", lambda: run_modes(binding, torch, W, N, args.mode, head, peaks))

    def orders():
        f32 = (extras.get("modes") or {}).get("fp32") or (head if args.mode == "fp32" else {})
        return run_orders(binding, torch, W, N, f32.get("kernel_ms"), f32.get("m2"))
    extra("orders", orders)
    extra("brickwork_dynamics", lambda: run_brickwork(binding, torch, W))
    extra("tfim_quench", lambda: run_tfim(binding, torch, W))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16_split": "f16x2-split (f32 accumulate)",
                  "bf16_split": "bf16x2-split (f32 accumulate)"}.get(args.mode, args.mode),
        "data": "synthetic",
        "config": {"workload": f"N={N} Haar-random state (complex64), all 4^{N} Pauli strings per step",
                   "N": N, "states_per_gpu": 1, "mode": args.mode, "l2_flush": "512 MiB write between steps",
                   "parallelism": f"replicas x{world}", "tuning": tuning,
                   "autotune_slice_ms": tune_ms},
        "m2": m2_val, "abs_diff_vs_oracle": (abs(m2_val - golden_m2(N, "complex64"))
                                             if golden_m2(N, "complex64") is not None else None),
        "states_per_s": world * args.steps / elapsed_s,
        "gpu_launches": int(launches), "wall_s": wall,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
    }
    loads = (extras.get("serving") or {}).get("loads") or {}
    mid = loads.get("0.5") or (next(iter(loads.values())) if loads else None)
    if mid and "server" in mid:
        line["serve_p50_ms"] = mid["server"]["p50_latency_ms"]
        line["serve_p99_ms"] = mid["server"]["p99_latency_ms"]
    line["extras"] = extras
    print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
