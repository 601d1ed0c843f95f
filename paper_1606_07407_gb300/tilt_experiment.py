"""Tilted lines on the worst case of two dimensions (Sec. 3.3, Alg. 3, Theorem 1), on the GPU.

Workload: batches of two-dimensional signals whose modes include the corners of axis-aligned
rectangles (inputs.draw_rectangle_signal), the configuration in which every projection onto an
axis puts each corner in a bin with another corner.  Each batch runs several ways on the same
signals: the parallel projections (lines along e_1 and e_2, coordinate shifts), which recover
no corner and stop at the round limit; Alg. 3's tilted lines with the triple given (in float
also with a floor on the prime rule); and, for context, the full unwrapping of Sec. 3.2
(u = (1, N)), which has no worst case in two dimensions.  Reported per (N, precision, form): the
share of signals recovered exactly, the largest round count, the mean samples per signal, and
modes recovered per second (wall time of one batched execute after warm-up, synchronised, the
median of the timed repeats).

Usage: python -m paper_1606_07407_gb300.tilt_experiment [--signals 256] [--repeats 5]
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import numpy as np

# (N, precision, triple with base > 2N and gcd(base, height) = 1, modes, rectangles, share of the
# signal count: the FP64 policy samples in double, whose pipe on this GPU is narrow)
CASES = ((512, "fp32", (1104, 47, 1105), 1000, 100, 1), (1024, "fp64", (2112, 65, 2113), 1000, 100, 8))


def _run(sfft, plans, sigs, handles, repeats, allow):
    batch = sfft.Batch(plans)
    res, sts, stats = batch.execute(handles, allow=allow)   # warm-up (and the result)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        batch.execute(handles, allow=allow)
        times.append(time.perf_counter() - t0)
    exact = 0
    for s, (f, a), st in zip(sigs, res, sts):
        gf, _ = sfft.sort_result(f.cpu().numpy(), a.cpu().numpy())
        if st == 0 and np.array_equal(gf, s.freqs[np.lexsort(s.freqs.T[::-1])]):
            exact += 1
    n = len(sigs)
    secs = statistics.median(times) if times else float("nan")
    return {"exact": exact / n, "rounds_max": stats["rounds"],   # batched stats: the longest signal's rounds
            "samples_mean": stats["samples"] / n, "seconds": secs,
            "modes_per_s": exact * sigs[0].k / secs if exact else 0.0}


def run(signals=256, repeats=5, seed=1606074071):
    import torch  # noqa: F401  (device memory for the binding)

    from . import sfft
    from .inputs import draw_rectangle_signal

    rows = []
    for N, prec, tilt, k, n_rect, div in CASES:
        n_sig = max(1, signals // div)
        sigs = [draw_rectangle_signal(N, k, n_rect, seed=seed + 31 * N + t) for t in range(n_sig)]
        handles = [sfft.Signal(s.freqs, s.coeffs, N) for s in sigs]
        forms = [("parallel", dict(blocks=(1, 1), max_rounds=24), (0, 2)),
                 ("tilt", dict(shift="tilt", tilt=tilt), (0,))]
        if prec == "fp32":
            # the rotated read-out resolves Q = (base + height) N values from one phase, so float
            # rounding of the bins matters (base + height) times more than for the coordinate
            # read-out; a floor on the prime raises a bin's magnitude (p |a|) above that rounding
            forms += [(f"tilt_pmin{q}", dict(shift="tilt", tilt=tilt, p_min=q), (0,)) for q in (256, 1024)]
        forms.append(("full_unwrap", dict(blocks=(2,)), (0,)))
        for name, kw, allow in forms:
            plans = [sfft.Plan(2, N, k, precision=prec, **kw)] * n_sig
            row = {"N": N, "precision": prec, "form": name, "k": k, "corners": 4 * n_rect, "signals": n_sig,
                   **({"tilt": list(tilt), "p_min": kw.get("p_min", 0)} if name.startswith("tilt") else {})}
            row.update(_run(sfft, plans, sigs, handles, repeats if name != "parallel" else 0, allow))
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--signals", type=int, default=256)
    ap.add_argument("--repeats", type=int, default=5)
    args = ap.parse_args(argv)
    run(args.signals, args.repeats)


if __name__ == "__main__":
    main()
