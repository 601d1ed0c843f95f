"""Prime schedules per signal class, from the measured table the autotuner writes.

Alg. 2 takes the prime factor c as an input (p = i-th prime >= c k*; c = 5 in the paper's
experiments) and leaves open how small the late rounds' primes may get.  Both shape the run:
c sets how many points a round samples against how many modes it leaves for later rounds, and a
floor p_min on the prime keeps late bins (p |a|) large against the float policies' rounding,
which matters once the read-out resolves many values from one phase (N up to 2^20); the
fused cut-over decides which rounds run one block per signal; and the width of the partial
unwrapping's blocks (Sec. 4.1) sets how many line directions there are, hence how many empty
rounds the stop rule waits for and how often two modes share a projected value.  The
autotuner (paper_1606_07407_gb300.autotune) measures candidates (c, p_min, cut-over, blocks) per class of
(d, N, k) on the GPU and keeps, per class, the fastest one that recovered every signal of its
training and validation batches exactly.  This module only reads that table.
"""
from __future__ import annotations

import hashlib
import json
import os

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_schedules.json")
DEFAULT = {"c": 5.0, "p_min": 0, "fuse_max_len": 0, "blocks": "narrow"}

_cache = None


def load_table(path: str = TABLE) -> dict:
    global _cache
    if path == TABLE and _cache is not None:
        return _cache
    try:
        with open(path) as fh:
            table = json.load(fh)
    except OSError:
        table = {"classes": []}
    if path == TABLE:
        _cache = table
    return table


def table_sha256(path: str = TABLE) -> str | None:
    try:
        with open(path, "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None


def class_of(entry: dict, d: int, N: int, k: int) -> bool:
    lg = int(N).bit_length() - 1
    return (entry["d"][0] <= d <= entry["d"][1] and entry["logN"][0] <= lg <= entry["logN"][1]
            and entry["k"][0] <= k <= entry["k"][1])


def schedule(d: int, N: int, k: int, table: dict | None = None) -> dict:
    """{"c": prime factor, "p_min": prime floor, "fuse_max_len": fused cut-over (0: the kernel's
    limit), "blocks": block rule ("narrow" or "wide", see inputs.blocks_for)} for a signal of
    dimension d, box side N and k modes: the first class of the table that holds it, else c = 5
    without a floor and the narrow blocks."""
    table = load_table() if table is None else table
    for entry in table.get("classes", []):
        if class_of(entry, d, N, k):
            return {"c": float(entry["c"]), "p_min": int(entry["p_min"]),
                    "fuse_max_len": int(entry.get("fuse_max_len", 0)), "blocks": entry.get("blocks", "narrow")}
    return dict(DEFAULT)
