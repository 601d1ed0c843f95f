"""Failure rate of the parallel projections against the bound of Sec. 4.2, on the GPU.

Sec. 4.2 bounds the probability that Alg. 2's parallel projections (a line along each block of a
partial unwrapping, Sec. 4.1) fail for k frequency vectors drawn uniformly from the N^d of the box:
1 - prod_{j=1..k} (N^d - (j - 1) sum_q N^{d_q}) / N^d, the probability that some vector lies on an
axis-parallel line (in the unwrapped coordinates) through an earlier one.  This module measures
the failure rate itself: batches of random signals run through the batched engine with the given
blocks, and a trial fails when the method stops at the round limit (status NOT_CONVERGED: some
modes share a bin with another mode on every block's line, whatever the prime).  Reported per
(d, N, blocks, k): trials, the failure share with its 95% Wilson interval, the mean count of
modes left unrecovered by a failing trial, the share of trials with a pair of vectors on a
common axis-parallel line (the event the bound covers, counted from the drawn vectors), the
bound, and the GPU wall time of the batch.

Usage: python -m paper_1606_07407_gb300.worst_case_experiment [--trials 4096]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

# (d, N, blocks, ks)
CASES = ((2, 32, (1, 1), (4, 8, 16, 32)),
         (3, 16, (1, 1, 1), (8, 32, 128)),
         (4, 8, (2, 2), (8, 32, 128)),
         (5, 1024, (3, 2), (1000,)))


def paper_bound(N: int, blocks, k: int) -> float:
    """Sec. 4.2's bound 1 - prod_j (N^d - (j - 1) sum_q N^{d_q}) / N^d (1 where a factor reaches 0)."""
    total = float(N) ** sum(blocks)
    line = sum(float(N) ** b for b in blocks)
    log_prod = 0.0
    for j in range(1, k + 1):
        f = (total - (j - 1) * line) / total
        if f <= 0.0:
            return 1.0
        log_prod += math.log(f)
    return 1.0 - math.exp(log_prod)


def pair_on_common_line(freqs: np.ndarray, N: int, blocks) -> bool:
    """Whether two vectors agree on every unwrapped block coordinate but one (a common line
    parallel to an axis of the unwrapped coordinates)."""
    starts = np.cumsum((0,) + tuple(blocks))[:-1]
    wt = np.stack([sum((freqs[:, b + r].astype(np.int64)) * N ** r for r in range(size))
                   for b, size in zip(starts, blocks)], axis=1)
    B = len(blocks)
    for q in range(B):
        rest = np.delete(wt, q, axis=1)
        if len({tuple(row) for row in rest.tolist()}) < len(rest):
            return True
    return False


def wilson(x: int, n: int, z: float = 1.96):
    if n == 0:
        return (0.0, 1.0)
    ph = x / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / den
    # the interval reaches 0 at x = 0 and 1 at x = n exactly (set them: rounding misses by an ulp)
    return (0.0 if x == 0 else max(0.0, c - h), 1.0 if x == n else min(1.0, c + h))


def run(trials=4096, seed=1606074072, max_rounds=40):
    import torch  # noqa: F401  (device memory for the binding)

    from . import sfft
    from .inputs import draw_signal

    rows = []
    for d, N, blocks, ks in CASES:
        for k in ks:
            T = trials if N ** d <= 1 << 20 else max(1, trials // 16)   # the full-size workload: fewer trials
            sigs = [draw_signal(d, N, k, seed=seed + 1000003 * d + 7919 * k + t) for t in range(T)]
            plans = [sfft.Plan(d, N, k, blocks=blocks, max_rounds=max_rounds)] * T
            batch = sfft.Batch(plans)
            handles = [sfft.Signal(s.freqs, s.coeffs, N) for s in sigs]
            t0 = time.perf_counter()
            res, sts, stats = batch.execute(handles, allow=(0, 2))
            secs = time.perf_counter() - t0
            fail = [i for i, st in enumerate(sts) if st == 2]
            left = [k - int(res[i][0].shape[0]) for i in fail]
            pairs = sum(pair_on_common_line(s.freqs, N, blocks) for s in sigs)
            lo, hi = wilson(len(fail), T)
            row = {"d": d, "N": N, "blocks": list(blocks), "k": k, "trials": T,
                   "fail": len(fail) / T, "fail_ci95": [lo, hi],
                   "left_per_fail": float(np.mean(left)) if left else 0.0,
                   "pair_event": pairs / T, "bound": paper_bound(N, blocks, k),
                   "other_status": sum(1 for st in sts if st not in (0, 2)), "seconds": secs}
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--trials", type=int, default=4096)
    args = ap.parse_args(argv)
    run(args.trials)


if __name__ == "__main__":
    main()
