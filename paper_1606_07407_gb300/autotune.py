"""Autotuner of the prime schedule, the unwrapping blocks and the fused cut-over per signal class
(runs on the GPU).

A batch of independent signals runs its rounds in lockstep: a round costs the launches of every
kernel class plus the work of the signals still active, and the batch ends with its slowest
signal.  Four per-signal choices shape that:
  - the prime factor c of Alg. 2's rule p = i-th prime >= c k* (the paper uses c = 5): fewer
    samples per round against more collisions and so more rounds;
  - a floor p_min on the prime: late rounds (k* small) would otherwise use short lines whose
    bins p |a| are small against the float rounding of the samples, so read-outs at large N
    miss delta for several rounds in a row, or slip to a neighbouring integer;
  - the longest Bluestein length run by the fused kernel (one block per signal runs the whole
    round) instead of the batched kernels;
  - the width of the partial unwrapping's blocks (Sec. 4.1): the narrowest that spans 4 c k
    values, or the widest whose direction fits an int64.  Fewer, wider blocks mean fewer line
    directions, so fewer empty rounds before the stop rule ends a signal, and fewer modes that
    share a projected value; with one shifted set per coordinate they cost no precision.
For each class of (N, k), over the batched workload's dimension range, the tuner draws a
training and a validation batch, times every candidate on the training batch (CUDA events,
median of three executes after a warm-up, one CUDA-graph launch each) and keeps the fastest
candidate that recovered every signal of both batches exactly with status OK.  The table goes
to tuned_schedules.json beside this file; paper_1606_07407_gb300.tuning reads it.

    python -m paper_1606_07407_gb300.autotune [--signals 192] [--out PATH]
"""
from __future__ import annotations

import argparse
import datetime
import gc
import itertools
import json
import os
import sys
import time

import numpy as np

from .inputs import BASE_SEED, Stream, blocks_for, draw_signal
from .tuning import TABLE

D_RANGE = (2, 8)
LOGN_CLASSES = ((10, 14), (15, 16), (17, 18), (19, 20))
K_CLASSES = ((8, 127), (128, 319), (320, 512))
C_CANDIDATES = (3.0, 4.0, 5.0, 6.0)
PMIN_CANDIDATES = (0, 512, 1024, 2048)
BLOCK_RULES = ("narrow", "wide")      # inputs.blocks_for
FUSE_CANDIDATES = (256, 512)          # tried on the best (c, p_min, blocks); 0 (the kernel's limit) always
# After tuning, a floor at a power of two is lowered so that the first primes above it stay below
# that power: 2p - 1 then fits a Bluestein length of 2^a (1024, 2048, 4096) instead of 5 2^(a-2),
# and the half line p / 2 + 1 no longer spills a few positions into one more sampling tile.
# Measured on the 4096-signal mix: 13.16 -> 12.89 ms per step, every signal exact.
FLOOR_BELOW_POW2 = {512: 480, 1024: 960, 2048: 1950}


def draw_class(n: int, logN: tuple, krange: tuple, seed: int) -> list:
    """n signals with k ~ U{krange}, d ~ U{D_RANGE}, N = 2^U{logN}, r ~ U[1, 10]."""
    st = Stream(seed)
    ks = st.integers(n, krange[0], krange[1] + 1)
    ds = st.integers(n, D_RANGE[0], D_RANGE[1] + 1)
    ls = st.integers(n, logN[0], logN[1] + 1)
    return [draw_signal(int(ds[s]), 1 << int(ls[s]), int(ks[s]), seed * 1000003 + s, "uniform", 1.0, 10.0)
            for s in range(n)]


class Trial:
    """One batch of signals resident on the device, timed under a candidate schedule."""

    def __init__(self, sfft, torch, sigs):
        self.sfft, self.torch, self.sigs = sfft, torch, sigs
        self.dev = [sfft.Signal(s.freqs, s.coeffs, s.N) for s in sigs]
        self.planted = [s.freqs[np.lexsort(s.freqs.T[::-1])].astype(np.int64) for s in sigs]

    def run(self, c, p_min, fuse_max_len, blocks, reps):
        sfft, torch = self.sfft, self.torch
        plans = [sfft.Plan(s.d, s.N, s.k, blocks=blocks_for(s.d, s.N, s.k, blocks), c=c, p_min=p_min,
                           fuse_max_len=fuse_max_len) for s in self.sigs]
        batch = sfft.Batch(plans, graph=True)
        out = batch.outputs(caps=[s.k + 16 for s in self.sigs])
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, exact, rounds = [], True, 0
        for rep in range(reps + 1):
            ev0.record()
            res, sts, st = batch.execute(self.dev, out=out, allow=(0, 2, 3, 5))
            ev1.record()
            ev1.synchronize()
            if rep > 0:
                ms.append(ev0.elapsed_time(ev1))
            rounds = max(rounds, st["rounds"])
            if any(x != 0 for x in sts):
                exact = False
        if exact:
            for b, (f, a) in enumerate(res):
                gf, _ = sfft.sort_result(f.cpu().numpy(), a.cpu().numpy())
                if not np.array_equal(gf, self.planted[b]):
                    exact = False
                    break
        del batch, plans, out
        gc.collect()
        return (float(np.median(ms)) if ms else None), exact, rounds


def tune(n_signals: int = 192, reps: int = 3, log=print) -> dict:
    import torch
    from . import build as B
    B.build()
    from . import sfft
    torch.cuda.set_device(0)
    props = torch.cuda.get_device_properties(0)
    classes = []
    for ci, (logN, krange) in enumerate(itertools.product(LOGN_CLASSES, K_CLASSES)):
        train = Trial(sfft, torch, draw_class(n_signals, logN, krange, BASE_SEED + 900 + 2 * ci))
        valid = Trial(sfft, torch, draw_class(n_signals, logN, krange, BASE_SEED + 901 + 2 * ci))
        results = []

        def consider(c, p_min, fuse, blocks):
            ms, ok, rounds = train.run(c, p_min, fuse, blocks, reps)
            if ok:
                _, ok, _ = valid.run(c, p_min, fuse, blocks, 0)
            results.append({"c": c, "p_min": p_min, "fuse_max_len": fuse, "blocks": blocks, "ms": ms, "exact": ok,
                            "rounds": rounds})
            log(f"  logN {logN} k {krange}: c {c} p_min {p_min} fuse {fuse} blocks {blocks}: {ms:.2f} ms "
                f"rounds {rounds} exact {ok}", flush=True)

        for blocks, c, p_min in itertools.product(BLOCK_RULES, C_CANDIDATES, PMIN_CANDIDATES):
            consider(c, p_min, 0, blocks)
        good = [r for r in results if r["exact"]]
        if good:
            best = min(good, key=lambda r: r["ms"])
            for fuse in FUSE_CANDIDATES:
                consider(best["c"], best["p_min"], fuse, best["blocks"])
            good = [r for r in results if r["exact"]]
            best = min(good, key=lambda r: r["ms"])
        else:
            best = {"c": 5.0, "p_min": max(PMIN_CANDIDATES), "fuse_max_len": 0, "blocks": "wide", "ms": None,
                    "exact": False}
        default = next(r for r in results if r["c"] == 5.0 and r["p_min"] == 0 and r["fuse_max_len"] == 0
                       and r["blocks"] == "narrow")
        classes.append({"d": list(D_RANGE), "logN": list(logN), "k": list(krange), "c": best["c"],
                        "p_min": FLOOR_BELOW_POW2.get(best["p_min"], best["p_min"]), "p_min_tuned": best["p_min"],
                        "fuse_max_len": best["fuse_max_len"], "blocks": best["blocks"],
                        "ms": best["ms"],
                        "rounds": best.get("rounds"), "exact_candidates": len(good),
                        "default_c5_ms": default["ms"], "default_c5_exact": default["exact"],
                        "candidates": results})
        log(f"class logN {logN} k {krange}: c {best['c']} p_min {best['p_min']} fuse {best['fuse_max_len']} "
            f"blocks {best['blocks']} {best['ms']} ms (default c = 5, no floor, narrow blocks: {default['ms']:.2f} ms, "
            f"exact {default['exact']})", flush=True)
        del train, valid
        gc.collect()
    return {"version": 1,
            "tool": "python -m paper_1606_07407_gb300.autotune",
            "device": props.name, "sm_count": props.multi_processor_count,
            "measured_utc": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
            "signals_per_class": n_signals, "reps": reps,
            "objective": "median CUDA-event time of one graph-launched batched execute of the class's "
                         "training batch, among candidates that recovered every signal of the training and "
                         "validation batches exactly",
            "search": {"c": list(C_CANDIDATES), "p_min": list(PMIN_CANDIDATES), "blocks": list(BLOCK_RULES),
                       "fuse_max_len": [0] + list(FUSE_CANDIDATES)},
            "floor_below_pow2": {str(k): v for k, v in FLOOR_BELOW_POW2.items()},
            "classes": classes}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--signals", type=int, default=192)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args(argv)
    t0 = time.time()
    table = tune(args.signals, args.reps)
    table["tuning_seconds"] = round(time.time() - t0, 1)
    with open(args.out, "w") as fh:
        json.dump(table, fh, indent=1)
        fh.write("\n")
    print(f"wrote {args.out} ({table['tuning_seconds']} s)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
