"""The precision study of the d = 20, N = 2^20 workload (|a| log-uniform in [1e-2, 1e2]), on the GPU.

Five arithmetic policies of the same method on the same signal:
  - fp64:          every step in double;
  - df64:          as fp64, the sampling in double-float (pairs of floats) on the FP32 pipe;
  - fp32:          float sampling and Bluestein DFT, phase ratio, read-out and coefficient in
                   double (the AUTO policy above N = 2^14);
  - fp32_bf16dft:  as fp32, with the DFT of rounds of p <= 8191 a split-BF16 tensor-core
                   contraction (FP32 accumulation) instead of Bluestein;
  - fp32_then_fp64: the fp32 rounds until a round accepts fewer than k* / 64 bins, then double
                   rounds continuing from the float registry.
For each: the exact-recovery rate (planted modes found / k), false positives (found modes not
planted), the relative coefficient error of the modes found against the planted values and
against a reference, status, rounds and GPU time of one execute.  At k = 100 000 the reference
is the fp64 arm (the CPU oracle would need about 2.4e12 sample terms); at k = 1000, the same
shape, the reference is the FP64 oracle (oracle/), whose own error against the planted values is
stated beside.

    python -m paper_1606_07407_gb300.precision_study [--k 100000] [--oracle-k 1000] [--json PATH]
        [--arms fp64,df64,...] [--no-graph]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from .inputs import WORKLOADS, draw_signal

ARMS = (("fp64", "all FP64"),
        ("df64", "double-float sampling on the FP32 pipe, FP64 DFT, ratio and read-out"),
        ("fp32", "FP32 sampling + Bluestein DFT, FP64 ratio"),
        ("fp32_bf16dft", "FP32 sampling, split-BF16 tensor-core DFT (p <= 8191) / FP32 Bluestein"),
        ("fp32_then_fp64", "FP32 rounds until they stall, then FP64 rounds from the float registry"))


def compare(freqs, coeffs, ref_freqs, ref_coeffs):
    """Modes in both sets: (count, max and median relative coefficient error against ref)."""
    ref = {tuple(w): a for w, a in zip(np.asarray(ref_freqs).tolist(), ref_coeffs)}
    rel = [abs(a - ref[tuple(w)]) / abs(ref[tuple(w)]) for w, a in zip(np.asarray(freqs).tolist(), coeffs)
           if tuple(w) in ref]
    if not rel:
        return 0, None, None
    return len(rel), float(np.max(rel)), float(np.median(rel))


def run_arm(sfft, torch, sig, blocks, prec, graph=True):
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=blocks, precision=prec, graph=graph)
    plan.execute(sfft.Signal(sig.freqs[:1], sig.coeffs[:1], sig.N), capacity=16, allow=(0, 2, 3, 5))   # warm-up
    dev = sfft.Signal(sig.freqs, sig.coeffs, sig.N)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    f, a, status, stats = plan.execute(dev, capacity=2 * sig.k + 16, allow=(0, 2, 3, 5))
    ev1.record()
    ev1.synchronize()
    gf, ga = sfft.sort_result(f.cpu().numpy(), a.cpu().numpy())
    return gf, ga, status, stats["rounds"], ev0.elapsed_time(ev1) / 1e3


def study(k: int, blocks, seed_offset: int, oracle: bool, arms=None, graph=True, log=print):
    import torch
    from . import build as B
    B.build()
    from . import sfft
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = draw_signal(wl.d, wl.N, k, wl.seed + seed_offset, wl.r_dist, wl.r_lo, wl.r_hi)
    planted_f = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
    planted_a = sig.coeffs[np.lexsort(sig.freqs.T[::-1])]
    planted = set(map(tuple, planted_f.tolist()))
    arms = list(arms or [a for a, _ in ARMS])
    results = {}
    for prec in arms:
        gf, ga, status, rounds, secs = run_arm(sfft, torch, sig, blocks, prec, graph)
        found = set(map(tuple, gf.tolist()))
        n_ok, emax, emed = compare(gf, ga, planted_f, planted_a)
        results[prec] = {"status": int(status), "rounds": int(rounds), "gpu_s": round(secs, 4),
                         "recovered": len(found & planted), "exact_rate": len(found & planted) / k,
                         "false_positives": len(found - planted),
                         "err_vs_planted_max": emax, "err_vs_planted_median": emed, "_f": gf, "_a": ga}
        log(f"  k={k} {prec}: status {status} rounds {rounds} {secs:.3f} s recovered {len(found & planted)}/{k} "
            f"false {len(found - planted)} err vs planted max {emax} median {emed}", flush=True)
    if oracle:
        import oracle.sfft_oracle as O
        t0 = time.perf_counter()
        ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, k, blocks, residual="bins", estimator="mean")
        oracle_s = time.perf_counter() - t0
        ref_f, ref_a = ref.freqs, ref.coeffs
        n_o, omax, omed = compare(ref_f, ref_a, planted_f, planted_a)
        results["oracle"] = {"converged": bool(ref.converged), "rounds": len(ref.rounds), "cpu_s": round(oracle_s, 1),
                             "recovered": len(set(map(tuple, ref_f.tolist())) & planted),
                             "err_vs_planted_max": omax, "err_vs_planted_median": omed}
        ref_name = "FP64 oracle"
    elif "fp64" in results:
        ref_f, ref_a, ref_name = results["fp64"]["_f"], results["fp64"]["_a"], "fp64 arm"
    else:
        ref_name = None
    for prec in arms:
        if ref_name:
            n_c, cmax, cmed = compare(results[prec]["_f"], results[prec]["_a"], ref_f, ref_a)
            results[prec].update(ref=ref_name, common_with_ref=n_c, err_vs_ref_max=cmax, err_vs_ref_median=cmed)
        del results[prec]["_f"], results[prec]["_a"]
    return {"d": sig.d, "N": sig.N, "k": k, "blocks": list(blocks), "r": "log-uniform [1e-2, 1e2]", "arms": results}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--k", type=int, default=100000)
    ap.add_argument("--oracle-k", type=int, default=1000)
    ap.add_argument("--json", default=None)
    ap.add_argument("--arms", default=",".join(a for a, _ in ARMS), help="comma-separated subset of the arms")
    ap.add_argument("--no-graph", action="store_true",
                    help="rounds enqueued from the host instead of a device-ended CUDA graph (for profilers)")
    args = ap.parse_args(argv)
    blocks = WORKLOADS["d20_N1048576_k100000"].blocks
    arms = [a for a in args.arms.split(",") if a]
    if any(a not in dict(ARMS) for a in arms):
        ap.error(f"arms must be among {[a for a, _ in ARMS]}")
    graph = not args.no_graph
    out = {"small": study(args.oracle_k, blocks, 100, oracle=True, arms=arms, graph=graph) if args.oracle_k > 0 else None,
           "full": study(args.k, blocks, 0, oracle=False, arms=arms, graph=graph) if args.k > 0 else None}
    text = json.dumps(out, indent=1)
    if args.json:
        with open(args.json, "w") as fh:
            fh.write(text + "\n")
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
