#!/usr/bin/env python
"""Benchmark of the sparse-FFT hot path: modes recovered per second at exact frequency recovery.

Default workload (mix4096): 4096 independent signals with k ~ U{8..512}, d ~ U{2..8},
N = 2^U{10..20}, r ~ U[1, 10], noiseless, each with its own plan (prime factor, prime floor,
fused cut-over and unwrapping-block rule from the tuned table of its (N, k) class), float
sampling and DFT with the phase ratio, read-out and coefficient in double above N = 2^14 (the
AUTO policy; --precision selects the others, among them df64: double-float sampling).  One step recovers all of them in one batched execute whose rounds run
as a CUDA graph with a device-ended while loop (the batched form); the plain form, one execute
per signal, is timed beside it on the same signals.  A step counts only if every recovered
frequency set equals the planted one.

Other workloads: the single-shape presets of paper_1606_07407_gb300.inputs.WORKLOADS, recovered
--batch signals at a time (batched) or one at a time (--form plain).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

if "--impl" in sys.argv and "reference" in sys.argv or "--cpu-baseline-only" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

from paper_1606_07407_gb300.inputs import BASE_SEED, WORKLOADS, batched_mix  # noqa: E402

METRIC = "modes recovered/s at exact freq recovery"
UNIT = "modes/s"
MIX = "mix4096"
MIX_SIGNALS = 4096
DEFAULT_WORKLOAD = MIX
FP32_ALU_LANES_PER_SM = 128      # FP32 FMA lanes per SM (Blackwell)
FP64_NOMINAL_TFLOPS = 1.25       # GB300's nominal FP64 rate (no measured figure is available)
ORACLE_TH = dict(tau=1e-3, rho=2.0 ** -17, delta=0.25)   # the float policies' default thresholds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# DRAM traffic per sampling launch, from the committed ncu summary of the d = 5 workload, valid
# while the sampling sources are the ones that summary was taken from
SAMPLE_PROFILE = os.path.join(ROOT, "profiles", "k_sample_d5_N1024_k1000_batch256.md")
SAMPLE_SOURCES = ["sample_tile.cuh", "engine_kernels.cuh", "engine.cuh", "sfft_internal.cuh"]


def sampling_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in SAMPLE_SOURCES:
        with open(os.path.join(ROOT, "paper_1606_07407_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def sample_traffic(workload: str):
    if workload != "d5_N1024_k1000":
        return None
    try:
        text = open(SAMPLE_PROFILE).read()
    except OSError:
        return None
    sha = re.search(r"sources_sha256:\s*([0-9a-f]{64})", text)
    val = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not sha or not val or sha.group(1) != sampling_sources_sha256():
        return None
    return float(val.group(1))


# ------------------------------------------------------------------ workloads

class Job:
    """The signals one rank recovers per step, with each signal's plan arguments."""

    def __init__(self, name: str, rank: int, batch: int, mix_signals: int = MIX_SIGNALS):
        from paper_1606_07407_gb300 import tuning
        self.name = name
        if name == MIX:
            from paper_1606_07407_gb300.inputs import blocks_for
            mix = batched_mix(mix_signals, seed=BASE_SEED + 4 + 1000 * rank)
            self.sigs = [s for s, _ in mix]
            self.sched = [tuning.schedule(s.d, s.N, s.k) for s in self.sigs]
            self.blocks = [blocks_for(s.d, s.N, s.k, sc["blocks"]) for s, sc in zip(self.sigs, self.sched)]
            self.homogeneous = False
            self.noise = 0.0
            self.table_sha = tuning.table_sha256()
        else:
            from paper_1606_07407_gb300 import dist as D
            wl = WORKLOADS[name]
            self.sigs = [wl.signal(seed_offset=o) for o in D.rank_seed_offsets(rank, batch)]
            self.blocks = [wl.blocks] * len(self.sigs)
            self.sched = [{"c": 5, "p_min": wl.p_min, "fuse_max_len": 0}] * len(self.sigs)
            self.homogeneous = True
            self.noise = wl.noise_sigma
            self.table_sha = None
        self.ks = [s.k for s in self.sigs]
        self.modes = int(sum(self.ks))

    def config(self) -> dict:
        if self.homogeneous:
            s = self.sigs[0]
            return {"workload": self.name, "d": s.d, "N": s.N, "k": s.k, "blocks": list(self.blocks[0]),
                    "signals_per_step": len(self.sigs), "p_min": self.sched[0]["p_min"]}
        ds = [s.d for s in self.sigs]
        ns = [s.N for s in self.sigs]
        cs = sorted({sc["c"] for sc in self.sched})
        pm = sorted({sc["p_min"] for sc in self.sched})
        return {"workload": self.name, "signals_per_step": len(self.sigs), "modes_per_step": self.modes,
                "k": [min(self.ks), max(self.ks)], "d": [min(ds), max(ds)], "N": [min(ns), max(ns)],
                "r": [1.0, 10.0],
                "schedule": f"per (N, k) class from the tuned table: prime factor c in {cs}, prime floor in {pm}, "
                            f"block rules {sorted({sc['blocks'] for sc in self.sched})} (narrow: the smallest b with "
                            f"N^b >= 4 c k; wide: the largest b with N^(b-1) in int64)",
                "tuned_table_sha256": self.table_sha}

    def make_plans(self, sfft, precision, residual, stream, graph=True):
        if self.homogeneous:
            s, sc = self.sigs[0], self.sched[0]
            plan = sfft.Plan(s.d, s.N, s.k, blocks=self.blocks[0], precision=precision, graph=graph, stream=stream,
                             residual=residual, noise_sigma=self.noise, p_min=sc["p_min"], c=sc["c"],
                             fuse_max_len=sc["fuse_max_len"])
            return [plan] * len(self.sigs)
        return [sfft.Plan(s.d, s.N, s.k, blocks=b, precision=precision, graph=graph, stream=stream,
                          residual=residual, p_min=sc["p_min"], c=sc["c"], fuse_max_len=sc["fuse_max_len"])
                for s, b, sc in zip(self.sigs, self.blocks, self.sched)]


def oracle_recover(sig, blocks, sched, residual):
    import oracle.sfft_oracle as O
    th = O.Thresholds(sigma=sig.noise_sigma, **ORACLE_TH)
    noise = None
    if sig.noise_sigma > 0:
        noise = lambda i, p, d, s=sig: O.black_box_noise(s.noise_seed, i, p, d, s.noise_sigma)  # noqa: E731
    return O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, blocks, th=th, residual=residual,
                              noise=noise, p_min=sched["p_min"], c=sched["c"], estimator="mean")


def oracle_throughput(workload: str, min_seconds: float, max_recoveries: int, seed_base: int,
                      residual: str = "bins", keep=None):
    """Runs the FP64 oracle on successive signals of the workload until min_seconds of CPU work
    (or max_recoveries), with the registry removed in the same form as the GPU arm and the same
    prime schedule.  For the mix, signal seed_base + n of rank 0's mix; else the preset's signal
    of that seed offset.  keep (a list), if given, receives (index, freqs, coeffs) of each.
    Returns (modes/s, recoveries, seconds, exact, modes)."""
    if workload == MIX:
        from paper_1606_07407_gb300 import tuning
        mix = batched_mix(MIX_SIGNALS, seed=BASE_SEED + 4)
    n, modes, t_total, exact = 0, 0, 0.0, True
    while n < max_recoveries and (t_total < min_seconds or n == 0):
        if workload == MIX:
            from paper_1606_07407_gb300.inputs import blocks_for
            sig, _ = mix[(seed_base + n) % MIX_SIGNALS]
            sched = tuning.schedule(sig.d, sig.N, sig.k)
            blocks = blocks_for(sig.d, sig.N, sig.k, sched["blocks"])
        else:
            wl = WORKLOADS[workload]
            sig, blocks, sched = (wl.signal(seed_offset=seed_base + n), wl.blocks,
                                  {"c": 5, "p_min": wl.p_min, "fuse_max_len": 0})
        t0 = time.perf_counter()
        res = oracle_recover(sig, blocks, sched, residual)
        t_total += time.perf_counter() - t0
        planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
        exact = exact and res.converged and np.array_equal(res.freqs, planted)
        if keep is not None:
            keep.append((seed_base + n, res.freqs, res.coeffs))
        n += 1
        modes += sig.k
    return modes / t_total, n, t_total, exact, modes


# Workloads whose single recovery takes the single-threaded oracle far longer than a bounded
# sample allows (about 5e9 and 2.4e12 sample terms): their CPU baseline is the oracle's sampling
# rate on a subset of round 1's points, converted to modes/s with the GPU run's own term count.
HEAVY = {"d10_N65536_k10000_noisy", "d20_N1048576_k100000"}


def oracle_term_rate(workload: str, seconds: float):
    """The oracle's black-box sampling (O.sample_sets) on round 1's line of the workload's first
    signal, over the first m points with m doubled until about `seconds` of work: sample terms
    per second and a description of the sample."""
    import oracle.sfft_oracle as O
    wl = WORKLOADS[workload]
    sig = wl.signal(seed_offset=0)
    p = O.ith_prime_at_least(1, max(5 * sig.k, wl.p_min))
    u = O.line_direction(sig.d, sig.N, wl.blocks, 1)
    m, t = 16, 0.0
    while True:
        t0 = time.perf_counter()
        O.sample_sets(sig.freqs, sig.coeffs, p, u, sig.N, x_values=np.arange(m))
        t = time.perf_counter() - t0
        if t >= seconds or m >= p:
            break
        m = min(p, 2 * m)
    terms = (sig.d + 1) * m * sig.k
    return terms / t, f"oracle sampling of {m} points x {sig.d + 1} sets x {sig.k} modes of round 1 ({t:.1f} s)"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append((time.perf_counter(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        if not inside and self.samples:
            mid = 0.5 * (t0 + t1)
            inside = [min(self.samples, key=lambda ts: abs(ts[0] - mid))[1]]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[0]) for s in inside if num(s[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": num(inside[0][1]), "reasons": reasons, "samples": len(inside)}


# ------------------------------------------------------------------ distributed helpers

def _dist_setup(n_gpus: int):
    from paper_1606_07407_gb300 import dist as D
    world, rank, local = D.world_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n_gpus > 0 else "gloo")
    return world, rank, local


def _barrier(world):
    from paper_1606_07407_gb300 import dist as D
    D.barrier()


def _max_over_ranks(world, value: float) -> float:
    from paper_1606_07407_gb300 import dist as D
    return D.max_over_ranks(value)


def _sum_over_ranks(world, value: float) -> float:
    from paper_1606_07407_gb300 import dist as D
    return D.sum_over_ranks(value)


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The FP64 oracle on the host, as it stands: each step recovers one signal of the workload
    (the mix: the next signal of rank 0's mix), single-threaded."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload in HEAVY:
        return run_reference_scaled(args)
    for w in range(args.warmup):
        oracle_throughput(args.workload, 0.0, 1, seed_base=10_000 + w, residual=args.residual)
    t, modes, exact = 0.0, 0, True
    for s in range(args.steps):
        _, n, secs, ok, m = oracle_throughput(args.workload, 0.0, 1, seed_base=s, residual=args.residual)
        t += secs
        modes += m
        exact = exact and ok
    value = modes / t if exact else 0.0
    cfg = {"workload": args.workload, "signals_per_step": 1, "form": "FP64 CPU oracle, one recovery per step",
           "residual": args.residual}
    if args.workload != MIX:
        wl = WORKLOADS[args.workload]
        cfg.update(d=wl.d, N=wl.N, k=wl.k, blocks=list(wl.blocks))
    else:
        cfg["sample"] = f"signals 0..{args.steps - 1} of the {MIX_SIGNALS}-signal mix, one per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded planted sparse signals)", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full recoveries, one per step, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_scaled(args):
    """The heavy workloads' reference arm: each step times the oracle's sampling of a bounded
    subset of round 1's points (as oracle_term_rate) and converts it with the sample terms of one
    recovery, (d + 1) x 6.1 k x k (the sum of the primes of a run, about 6.1 k at c = 5, times the
    modes summed per point): an estimate of a full recovery that flatters the oracle (its DFT and
    classification are left out)."""
    wl = WORKLOADS[args.workload]
    terms_per_rec = (wl.d + 1) * 6.1 * max(wl.k, wl.p_min / 5) * wl.k
    secs = max(1.0, args.cpu_seconds / max(args.steps, 1))
    for _ in range(args.warmup):
        oracle_term_rate(args.workload, 0.2)
    rates = [oracle_term_rate(args.workload, secs) for _ in range(args.steps)]
    rate = float(np.mean([r for r, _ in rates]))
    value = wl.k * rate / terms_per_rec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl.k / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded planted sparse signals)",
        "config": {"workload": args.workload, "d": wl.d, "N": wl.N, "k": wl.k, "blocks": list(wl.blocks),
                   "form": "FP64 CPU oracle sampling rate on a bounded sample, scaled to one recovery"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": rates[-1][1] + f", scaled by {terms_per_rec:.3g} terms per recovery"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def _timed_steps(torch, stream, flush, steps, step_fn):
    """Runs `steps` steps, each bracketed by CUDA events on the launch stream, with an L2
    flush (a 256 MiB write) before each step outside the events.  Returns ms per step and
    the per-step results."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms, outs = [], []
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        outs.append(step_fn())
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    return ms, outs


def _precision_name(prec: str) -> str:
    return {"fp32": "AUTO: float sampling and DFT; phase ratio, read-out and coefficient in double above N = 2^14",
            "fp32_fp64ratio": "float sampling and DFT; phase ratio, read-out and coefficient in double",
            "fp32_only": "every step in float",
            "fp64": "every step in double",
            "fp32_bf16dft": "as AUTO, with the DFT of rounds of p <= 8191 a split-BF16 tensor-core contraction "
                            "(FP32 accumulate)",
            "df64": "double engine with sampling in double-float (pairs of floats on the FP32 pipe, about 48 "
                    "significant bits); DFT, phase ratio, read-out and coefficient in double"}[prec]


def df64_ops_per_term(d: int) -> float:
    """FP32 operations the double-float sampler spends per term (set x mode x sample): per mode,
    row pair and lane it forms E = U L (two products of 4 operations, two accumulations of 12)
    once for the NS sets of its group, then 4 multiply-accumulates of 12 operations per set, and
    the pair serves two samples.  NS is the set group's size for the d + 1 sets."""
    ns = d + 1
    groups = -(-ns // 8)
    gsize = -(-ns // groups)
    return (4 * 12 + 32.0 / gsize) / 2.0


def run_ours(args):
    import torch
    world, rank, local = _dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_1606_07407_gb300 import build as B
    if rank == 0:
        B.build()
    _barrier(world)
    from paper_1606_07407_gb300 import sfft

    job = Job(args.workload, rank, args.batch, args.signals)
    stream = torch.cuda.current_stream()
    nb = len(job.sigs)
    # inputs resident in HBM before timing
    dev = [sfft.Signal(s.freqs, s.coeffs, s.N, noise_sigma=s.noise_sigma, noise_seed=s.noise_seed) for s in job.sigs]
    planted = [s.freqs[np.lexsort(s.freqs.T[::-1])].astype(np.int64) for s in job.sigs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    t_plan0 = time.perf_counter()
    plans = job.make_plans(sfft, args.precision, args.residual, stream)
    batch = sfft.Batch(plans, graph=True, stream=stream)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t_plan0
    caps = [k + 16 for k in job.ks]
    bout = batch.outputs(caps=caps)   # room for the recovered set (overflow: CAPACITY)
    allow = (0, 2, 3, 5)

    def step_batched():
        res, sts, st = batch.execute(dev, out=bout, allow=allow)
        return sts, st, res

    pouts = [(torch.empty((2 * k + 16, s.d), dtype=torch.int32, device="cuda"),
              torch.empty((2 * k + 16,), dtype=torch.complex128, device="cuda")) for k, s in zip(job.ks, job.sigs)]

    def step_plain():
        sts, res, st = [], [], None
        for b in range(nb):
            f, a, status, st = plans[b].execute(dev[b], capacity=2 * job.ks[b] + 16, out=pouts[b], allow=allow)
            sts.append(status)
            res.append((f, a))
        return sts, st, res

    head_fn = step_batched if args.form == "batched" else step_plain
    for _ in range(args.warmup):
        head_fn()
    torch.cuda.synchronize()

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except (ValueError, IndexError):
            gpu_index = local
    sampler = ClockSampler(gpu_index) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    _barrier(world)
    torch.cuda.synchronize()
    t_host0 = time.perf_counter()
    step_ms, outs = _timed_steps(torch, stream, flush, args.steps, head_fn)
    torch.cuda.synchronize()
    t_host1 = time.perf_counter()
    _barrier(world)
    clocks = sampler.summary(t_host0, t_host1) if sampler else None
    if sampler:
        sampler.stop()

    # every step's statuses, and the last step's sets element by element against the planted ones
    ok_all = all(all(x == 0 for x in sts) for sts, _, _ in outs)
    last = [sfft.sort_result(f.cpu().numpy(), a.cpu().numpy()) for f, a in outs[-1][2]]
    exact_slots = sum(1 for b, (gf, _) in enumerate(last) if np.array_equal(gf, planted[b]))
    ok_all = ok_all and exact_slots == nb
    total_ms = _max_over_ranks(world, float(sum(step_ms)))
    modes = _sum_over_ranks(world, float(args.steps * job.modes)) if ok_all else 0.0
    value = modes / (total_ms / 1e3)
    launches_step = outs[-1][1]["launches"] if args.form == "batched" else None
    gpu_launches = int(sum(sum(st["launches"].values()) for _, st, _ in outs)) if args.form == "batched" else \
        int(args.steps * nb * sum(outs[-1][1]["launches"].values()))
    rounds_step = outs[-1][1]["rounds"] if args.form == "batched" else None

    # the other form, on the same signals, for comparison
    other_fn = step_plain if args.form == "batched" else step_batched
    other_ms, other_value = [], None
    if args.other_steps > 0:
        other_fn()
        other_ms, other_outs = _timed_steps(torch, stream, flush, args.other_steps, other_fn)
        other_ok = all(all(x == 0 for x in sts) for sts, _, _ in other_outs)
        other_value = (args.other_steps * job.modes) / (sum(other_ms) / 1e3) if other_ok else 0.0

    # profiled pass (same batch, rounds enqueued from the host with CUDA events around each
    # kernel class on the launch stream): kernel shares and the sampling kernel's roofline
    pbatch = sfft.Batch(plans, graph=False, profile=True, stream=stream)
    pout = pbatch.outputs(caps=caps)
    pbatch.execute(dev, out=pout, allow=allow)
    prof_ms, prof = _timed_steps(torch, stream, flush, args.profile_steps,
                                 lambda: pbatch.execute(dev, out=pout, allow=allow))
    pstats = [o[2] for o in prof]
    # terms the batched sampling kernel summed (the fused kernel samples the short rounds)
    terms = sum(st["terms"] - st["terms_fused"] for st in pstats)
    sample_ms = sum(st["kernel_ms"]["sample"] for st in pstats)
    class_ms = {k: sum(st["kernel_ms"][k] for st in pstats) for k in sfft.KCLASSES}
    sample_launches = sum(st["launches"]["sample"] for st in pstats)
    flops = 8.0 * terms                      # one complex multiply-add (4 FMA) per term
    achieved = flops / (sample_ms / 1e3) / 1e12 if sample_ms > 0 else 0.0
    props = torch.cuda.get_device_properties(local)
    sm_max = (clocks or {}).get("sm_max_mhz") or _peaks().get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * FP32_ALU_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peak_basis = f"{props.multi_processor_count} SMs x {FP32_ALU_LANES_PER_SM} FP32 FMA lanes x 2 x {sm_max:.0f} MHz"
    if args.precision == "fp64":
        peak = FP64_NOMINAL_TFLOPS
        peak_basis = ("GB300's nominal FP64 rate; the paired evaluation executes 4 of the 8 algorithmic flops of a "
                      "term, so the fraction can exceed 1")
    elif args.precision == "df64":
        ops = df64_ops_per_term(job.sigs[0].d)
        peak = props.multi_processor_count * FP32_ALU_LANES_PER_SM * sm_max * 1e6 * 8.0 / ops / 1e12
        peak_basis = (f"double-float peak: {props.multi_processor_count} SMs x {FP32_ALU_LANES_PER_SM} FP32 lanes x "
                      f"{sm_max:.0f} MHz FP32 operations/s x 8 algorithmic flops per term / {ops:.2f} FP32 operations "
                      f"per term of the double-float sampler")
    tot_class = sum(class_ms.values())
    del pbatch, pout

    # end to end through the public API with host buffers: per step, the step's inputs (all
    # signals' modes, packed) copied pinned host -> device, the signal handles refilled in place by
    # one call, recovery, device -> host of the results.  The steps are pipelined over a second
    # stream: step i + 1's inputs and step i - 1's results cross PCIe/C2C while step i recovers
    # (double-buffered inputs and outputs); the wall clock runs from the first copy to the last.
    host_fw = torch.from_numpy(np.concatenate([s.freqs.astype(np.int32).reshape(-1) for s in job.sigs])).pin_memory()
    host_ca = torch.from_numpy(np.concatenate([s.coeffs.astype(np.complex128) for s in job.sigs])).pin_memory()
    dev_in = [(torch.empty_like(host_fw, device="cuda"), torch.empty_like(host_ca, device="cuda")) for _ in range(2)]
    h2d = host_fw.numel() * 4 + host_ca.numel() * 16
    outs2 = [bout, batch.outputs(caps=caps)]
    host_out = [(torch.empty(o[1].shape, dtype=torch.int32).pin_memory(),
                 torch.empty(o[2].shape, dtype=torch.complex128).pin_memory()) for o in outs2]
    d2h = host_out[0][0].numel() * 4 + host_out[0][1].numel() * 16
    copy_stream = torch.cuda.Stream()
    in_ready = [torch.cuda.Event() for _ in range(2)]

    def h2d_step(i):
        with torch.cuda.stream(copy_stream):
            fw, ca = dev_in[i % 2]
            fw.copy_(host_fw, non_blocking=True)
            ca.copy_(host_ca, non_blocking=True)
            in_ready[i % 2].record(copy_stream)

    def d2h_step(i):
        copy_stream.wait_stream(stream)   # the step's results are written (execute has returned)
        with torch.cuda.stream(copy_stream):
            host_out[i % 2][0].copy_(outs2[i % 2][1], non_blocking=True)
            host_out[i % 2][1].copy_(outs2[i % 2][2], non_blocking=True)

    e2e_ok = True
    e2e_checks = []   # each step's statuses and counts, verified after the clock stops
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d_step(0)
    for i in range(args.e2e_steps):
        if i + 1 < args.e2e_steps:
            h2d_step(i + 1)
        flush.zero_()
        stream.wait_event(in_ready[i % 2])
        fw, ca = dev_in[i % 2]
        sfft.assign_many(dev, fw, ca, job.ks, stream=stream)
        res, sts, _ = batch.execute(dev, out=outs2[i % 2], allow=allow)
        d2h_step(i)
        e2e_checks.append((sts, res.n_found))
    copy_stream.synchronize()
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0)
    for sts, nf in e2e_checks:
        e2e_ok = e2e_ok and all(x == 0 for x in sts) and all(int(n) == k for n, k in zip(nf, job.ks))
    e2e_ms = _max_over_ranks(world, e2e_ms)
    e2e_modes = _sum_over_ranks(world, float(args.e2e_steps * job.modes)) if e2e_ok else 0.0
    e2e_value = e2e_modes / (e2e_ms / 1e3)

    if rank != 0:
        return 0
    cfg = job.config()
    cfg.update({
        "form": ("batched: all signals in every launch, device-ended CUDA-graph round loop"
                 if args.form == "batched" else "plain: one signal per execute, CUDA-graph round loop"),
        "precision": _precision_name(args.precision),
        "residual": ("registry removed bin by bin after the DFT" if args.residual == "bins"
                     else "registry sampled with the black box (f - g)"),
        "l2": "flushed between timed steps (256 MiB write)", "exact_recovery": bool(ok_all),
        "exact_slots": f"{exact_slots}/{nb}",
        "plan_time_s": round(plan_s, 3),
        "plan_time_note": "plans and the batch are made before timing: device buffers, prime tables, and "
                          "round 1's root tables and Bluestein filter spectra (fixed by k) live with them"})
    if rounds_step is not None:
        cfg["rounds_last_step"] = rounds_step
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "df64": "df64"}.get(args.precision, "fp32"),
        "data": "synthetic (seeded planted sparse signals, resident in HBM)",
        "config": cfg,
        "other_form": {"form": "plain" if args.form == "batched" else "batched", "value": other_value,
                       "unit": UNIT, "steps": args.other_steps,
                       "ms_per_step": sum(other_ms) / max(len(other_ms), 1),
                       "batched_over_plain": (value / other_value if other_value else None)
                       if args.form == "batched" else None},
        "roofline": {"bound": "alu", "kernel": "k_sample", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": sample_traffic(args.workload),
                     "peak_basis": peak_basis,
                     "measured": f"CUDA events around each sampling launch, {args.profile_steps} profiled steps "
                                 "of the same batch (rounds enqueued from the host); terms of the rounds "
                                 "the batched kernels ran, 8 flops each",
                     "launches": sample_launches,
                     "avg_launch_us": 1e3 * sample_ms / max(sample_launches, 1),
                     "profiled_ms_per_step": sum(prof_ms) / max(len(prof_ms), 1)},
        "kernel_share": {k: round(v / tot_class, 4) if tot_class else None for k, v in class_ms.items()},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": args.e2e_steps,
                "form": "public API (assign_many + batch execute), host buffers, copies of step i+1 / i-1 "
                        "overlapping step i on a second stream, L2 flushed before each step (inside the clock)"},
    }
    if launches_step is not None:
        line["launches_per_step"] = launches_step
    if world == 1 and not args.no_cpu_baseline:
        if args.workload in HEAVY:
            # terms of one recovery, from the last timed step (all signals of a step are alike)
            terms_per_rec = float(outs[-1][1]["terms"]) / (nb if args.form == "batched" else 1)
            cb = cpu_baseline_scaled(args, terms_per_rec, job.sigs[0].k)
            line["cpu_baseline"] = cb
            line["precision_report"] = {"exact_sets_vs_planted": f"{exact_slots}/{nb}",
                                        "oracle_signals": 0, "note": "a full oracle recovery of this workload is "
                                        "beyond a bounded CPU sample"}
        else:
            cb, ref = cpu_baseline(args)
            line["cpu_baseline"] = cb
            line["precision_report"] = precision_report(ref, last, planted, job)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def precision_report(ref, last, planted, job):
    """Every recovered set against the planted one, and the coefficients of the signals the
    oracle recovered (the cpu_baseline sample) against the FP64 oracle's."""
    rel = []
    same = 0
    ref = [(idx, rf, ra) for idx, rf, ra in ref if idx < len(last)]
    for idx, rf, ra in ref:
        gf, ga = last[idx]
        if np.array_equal(gf, rf):
            same += 1
            rel.append(np.abs(ga - ra) / np.abs(ra))
    rel = np.concatenate(rel) if rel else np.zeros(0)
    return {"exact_sets_vs_planted": f"{sum(1 for b, (gf, _) in enumerate(last) if np.array_equal(gf, planted[b]))}"
                                     f"/{len(last)}",
            "oracle_signals": len(ref), "sets_equal_oracle": f"{same}/{len(ref)}",
            "coeff_rel_err_vs_oracle": {"max": float(rel.max()) if rel.size else None,
                                        "median": float(np.median(rel)) if rel.size else None,
                                        "modes": int(rel.size)}}


def cpu_baseline(args):
    """The oracle, single-threaded, in a child process on a bounded sample of the workload; then
    one oracle process per host core on independent signals (their summed rates under
    all_cores).  Also returns the sample's oracle results [(index, freqs, coeffs)]."""
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "oracle.npz")
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--workload", args.workload,
               "--cpu-seconds", str(args.cpu_seconds), "--residual", args.residual, "--cpu-all-cores",
               "--oracle-out", out]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            cb = json.loads(r.stdout.strip().splitlines()[-1])
        except Exception as exc:  # noqa: BLE001
            return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}, []
        ref = []
        if os.path.exists(out):
            z = np.load(out)
            for i in range(int(z["n"])):
                ref.append((int(z[f"idx{i}"]), z[f"w{i}"], z[f"a{i}"]))
        return cb, ref


def cpu_baseline_scaled(args, terms_per_recovery: float, k: int):
    """The heavy workloads' CPU baseline: the oracle's sampling rate (one thread, in a child
    process) times the GPU run's terms per recovery, as modes/s.  The oracle's DFT and
    classification are left out, which only flatters it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--workload", args.workload,
           "--cpu-seconds", str(args.cpu_seconds)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as exc:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}
    rate = d["terms_per_s"]
    return {"value": k * rate / terms_per_recovery, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": d["sample"] + f"; {rate:.3g} terms/s scaled by the {terms_per_recovery:.3g} sample terms of one "
                                    f"GPU recovery (the oracle's DFT and classification not counted)"}


def _oracle_worker(workload, seconds, seed_base, residual):
    return oracle_throughput(workload, seconds, 1000, seed_base=seed_base, residual=residual)


def oracle_all_cores(workload, seconds, residual):
    """One single-threaded oracle process per available core (spawned: no state is inherited),
    each on its own signals for about `seconds`; the aggregate rate is the sum of the processes'
    rates, each over its own recoveries' time (process start-up is not counted)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    stride = 7 if workload == MIX else 100_000
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(workload, seconds, stride * (i + 1) + (50 if workload == MIX else 0),
                                             residual) for i in range(cores)])
    exact = all(r[3] for r in res)
    return {"value": sum(r[0] for r in res) if exact else 0.0, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {min(r[1] for r in res)}-{max(r[1] for r in res)} full recoveries "
                      f"(about {seconds:.0f} s each, one thread each, residual {residual})"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + [MIX])
    ap.add_argument("--batch", type=int, default=256, help="signals recovered per step (single-shape presets)")
    ap.add_argument("--signals", type=int, default=MIX_SIGNALS,
                    help="signals of the mix, drawn the same way (fewer: a smaller case for profiling)")
    ap.add_argument("--form", default="batched", choices=["batched", "plain"])
    ap.add_argument("--other-steps", type=int, default=1)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_fp64ratio", "fp32_only", "fp64",
                                                           "fp32_bf16dft", "df64"],
                    help="fp32: AUTO (ratio in double above N = 2^14); fp32_fp64ratio: ratio always in double")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-baseline-only", action="store_true")
    ap.add_argument("--cpu-all-cores", action="store_true",
                    help="with --cpu-baseline-only: also time one oracle process per host core")
    ap.add_argument("--oracle-out", default=None, help="with --cpu-baseline-only: save the oracle's results (npz)")
    ap.add_argument("--residual", default="bins", choices=["bins", "samples"],
                    help="registry removed from the transform bin by bin, or sampled with the black box")
    args = ap.parse_args(argv)
    if args.cpu_baseline_only and args.workload in HEAVY:
        rate, what = oracle_term_rate(args.workload, args.cpu_seconds)
        print(json.dumps({"terms_per_s": rate, "sample": what}))
        return 0
    if args.cpu_baseline_only:
        keep = []
        v, n, secs, exact, modes = oracle_throughput(args.workload, args.cpu_seconds, 1000, seed_base=0,
                                                     residual=args.residual, keep=keep)
        what = f"signals 0..{n - 1} of the mix" if args.workload == MIX else f"{n} signals of the workload"
        out = {"value": v if exact else 0.0, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} full recoveries ({what}, {modes} modes, {secs:.1f} s, single thread, "
                         f"residual {args.residual})"}
        if args.oracle_out:
            arrs = {"n": np.array(len(keep))}
            for i, (idx, w, a) in enumerate(keep):
                arrs[f"idx{i}"], arrs[f"w{i}"], arrs[f"a{i}"] = np.array(idx), w, a
            np.savez(args.oracle_out, **arrs)
        if args.cpu_all_cores:
            try:
                out["all_cores"] = oracle_all_cores(args.workload, max(1.0, args.cpu_seconds * 2 / 3), args.residual)
            except Exception as exc:  # noqa: BLE001
                out["all_cores"] = {"value": None, "sample": f"failed: {exc}"}
        print(json.dumps(out))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
