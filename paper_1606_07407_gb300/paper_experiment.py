"""The paper's own experiment (Sec. 5): Alg. 2 as printed on d = 100 and 1000 variables.

Setup of Sec. 5: N = 20 per coordinate, blocks of d1 = 5 coordinates (d2 = d / 5 blocks), the
box [-N/2, N/2)^d, coefficients of modulus 1 with uniform phases, c = 5, shifts
eps = 1 / (2 N^{d1}) along each block's unwrap vector, k = 2^0 .. 2^10 and 100 trials per
(d, k).  The trials of one (d, k) run as one batched execute in FP64 (the block read-out
resolves N^5 = 3.2e6 values from one phase).  Reported per (d, k), as in Fig. 4-5: the share
of trials whose recovered set is the planted one, the mean and largest l2 norm of the
coefficient error, and the mean number of samples, also divided by d k (Theorem 3: Theta(d k)).
The paper's figure values are not in its source, so there is nothing to compare against
beyond its claims: exact frequencies, errors at double round-off, samples growing like d k.

Usage: python -m paper_1606_07407_gb300.paper_experiment [--trials 100] [--dims 100 1000]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(dims=(100, 1000), ks=tuple(2 ** e for e in range(11)), trials=100, seed=1606074070):
    import torch  # noqa: F401  (device memory for the binding)

    from . import sfft
    from .inputs import draw_signal

    rows = []
    for d in dims:
        blocks = (5,) * (d // 5)
        for k in ks:
            sigs = [draw_signal(d, 20, k, seed=seed + 7919 * d + 104729 * k + t, box_lo=-10, unit_modulus=True)
                    for t in range(trials)]
            plan = sfft.Plan(d, 20, k, blocks=blocks, precision="fp64", shift="block", box_lo=-10)
            batch = sfft.Batch([plan] * trials)
            handles = [sfft.Signal(s.freqs, s.coeffs, 20) for s in sigs]
            t0 = time.perf_counter()
            res, sts, stats = batch.execute(handles, allow=(0, 2, 3, 5))
            secs = time.perf_counter() - t0
            exact, l2, samples = 0, [], []
            for s, (f, a), st in zip(sigs, res, sts):
                gf, ga = sfft.sort_result(f.cpu().numpy(), a.cpu().numpy())
                order = np.lexsort(s.freqs.T[::-1])
                if st == 0 and np.array_equal(gf, s.freqs[order]):
                    exact += 1
                    l2.append(float(np.linalg.norm(ga - s.coeffs[order])))
            # batched stats hold totals over the slots: samples per trial is their mean
            samples = stats["samples"] / trials
            rows.append({"d": d, "k": k, "trials": trials, "exact": exact / trials,
                         "l2_mean": float(np.mean(l2)) if l2 else None,
                         "l2_max": float(np.max(l2)) if l2 else None,
                         "samples_mean": samples, "samples_per_dk": samples / (d * k), "seconds": secs})
            print(json.dumps(rows[-1]), flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--trials", type=int, default=100)
    ap.add_argument("--dims", type=int, nargs="+", default=[100, 1000])
    ap.add_argument("--kmax-exp", type=int, default=10)
    args = ap.parse_args(argv)
    run(tuple(args.dims), tuple(2 ** e for e in range(args.kmax_exp + 1)), args.trials)


if __name__ == "__main__":
    main()
