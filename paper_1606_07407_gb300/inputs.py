"""Seeded synthetic inputs for the sparse-FFT hot path.

This module only draws inputs: the planted frequency vectors and coefficients of
a synthetic black-box signal f(t) = sum_j a_j exp(2 pi i w_j . t) (Sec. 2.2,
Eq. 9 / Eq. 32), and the workload presets.  It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any step of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here from its
published definition so that the stream is identical on every machine and
numpy version: output i of a stream seeded with s is mix(s + (i+1) * gamma).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

#: seed of workload preset c is BASE_SEED + c (the paper's arXiv id).
BASE_SEED = 1606074070


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential reader of one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & _MASK64
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi) (floor of a 53-bit uniform times the range)."""
        span = hi - lo
        return (np.floor(self.uniform(n) * span).astype(np.int64) + lo)


@dataclass
class Signal:
    """One planted sparse signal: k distinct frequency vectors and coefficients."""
    d: int
    N: int
    freqs: np.ndarray          # int32 [k, d], each coordinate in [box_lo, box_lo + N)
    coeffs: np.ndarray         # complex128 [k]
    box_lo: int = 0            # 0 for [0, N)^d, -N/2 for the paper's [-N/2, N/2)^d
    noise_sigma: float = 0.0
    noise_seed: int = 0

    @property
    def k(self) -> int:
        return int(self.freqs.shape[0])


def draw_signal(d: int, N: int, k: int, seed: int, r_dist: str = "uniform",
                r_lo: float = 1.0, r_hi: float = 2.0, box_lo: int = 0,
                noise_sigma: float = 0.0, unit_modulus: bool = False) -> Signal:
    """Draw k distinct frequency vectors uniformly from the box and coefficients
    a = r exp(i theta), theta ~ U[0, 2 pi), r ~ U[r_lo, r_hi] ("uniform") or
    log-uniform on [r_lo, r_hi] ("loguniform"); unit_modulus forces r = 1."""
    if k < 0 or d < 1 or N < 2:
        raise ValueError("bad signal shape")
    if k > N ** d:
        raise ValueError("k exceeds the number of frequency vectors in the box")
    st = Stream(seed)
    seen: set[bytes] = set()
    rows: list[np.ndarray] = []
    while len(rows) < k:
        need = k - len(rows)
        cand = st.integers(need * d, 0, N).reshape(need, d)
        for row in cand:
            key = row.tobytes()
            if key not in seen:          # distinct frequencies: duplicates are redrawn
                seen.add(key)
                rows.append(row)
    freqs = (np.array(rows, dtype=np.int64).reshape(k, d) + box_lo).astype(np.int32)
    u_r = st.uniform(k)
    u_t = st.uniform(k)
    if unit_modulus:
        r = np.ones(k)
    elif r_dist == "uniform":
        r = r_lo + (r_hi - r_lo) * u_r
    elif r_dist == "loguniform":
        r = np.exp(math.log(r_lo) + (math.log(r_hi) - math.log(r_lo)) * u_r)
    else:
        raise ValueError(r_dist)
    coeffs = r * np.exp(2j * np.pi * u_t)
    return Signal(d=d, N=N, freqs=freqs, coeffs=coeffs.astype(np.complex128), box_lo=box_lo,
                  noise_sigma=noise_sigma, noise_seed=(seed * 7919 + 17) & _MASK64)


def draw_rectangle_signal(N: int, k: int, n_rect: int, seed: int, r_lo: float = 1.0, r_hi: float = 10.0) -> Signal:
    """A two-dimensional signal of k distinct modes in [0, N)^2 whose first 4 n_rect modes are
    the corners of n_rect axis-aligned rectangles (distinct corners; two x and two y values
    each), the rest drawn uniformly; coefficients r exp(i theta), r ~ U[r_lo, r_hi].  Every
    corner shares its first coordinate with one corner and its second with another, the
    configuration that defeats the projections onto the axes (the worst case of the tilted
    lines' section of the paper)."""
    if 4 * n_rect > k or k > N * N or N < 2:
        raise ValueError("bad rectangle signal shape")
    st = Stream(seed)
    seen: set = set()
    rows: list = []
    while len(rows) < 4 * n_rect:
        x0, x1, y0, y1 = (int(v) for v in st.integers(4, 0, N))
        if x0 == x1 or y0 == y1:
            continue
        corners = [(x0, y0), (x0, y1), (x1, y0), (x1, y1)]
        if any(c in seen for c in corners):
            continue
        seen.update(corners)
        rows.extend(corners)
    while len(rows) < k:
        x, y = (int(v) for v in st.integers(2, 0, N))
        if (x, y) not in seen:
            seen.add((x, y))
            rows.append((x, y))
    freqs = np.array(rows, dtype=np.int32).reshape(k, 2)
    r = r_lo + (r_hi - r_lo) * st.uniform(k)
    coeffs = r * np.exp(2j * np.pi * st.uniform(k))
    return Signal(d=2, N=N, freqs=freqs, coeffs=coeffs.astype(np.complex128))


@dataclass
class Workload:
    """A workload preset: signal shape, line-direction blocks and precision policy."""
    name: str
    d: int
    N: int
    k: int
    blocks: tuple
    r_dist: str = "uniform"
    r_lo: float = 1.0
    r_hi: float = 10.0
    noise_sigma: float = 0.0
    seed: int = BASE_SEED
    p_min: int = 0          # floor of the prime schedule the workload is run with (0: none)
    extra: dict = field(default_factory=dict)

    def signal(self, seed_offset: int = 0) -> Signal:
        return draw_signal(self.d, self.N, self.k, self.seed + seed_offset, self.r_dist,
                           self.r_lo, self.r_hi, noise_sigma=self.noise_sigma)


#: Workload presets shaped like the paper's experiments (Sec. 5) and the five
#: hot-path configurations: (1) d=2 plain, (2) d=5 higher dimension, (3) d=10
#: noisy, (5) d=20 precision stress.  The batched mix (4) is drawn by
#: ``batched_mix``.
WORKLOADS = {
    "d2_N1024_k16": Workload("d2_N1024_k16", 2, 1024, 16, (1, 1), r_lo=1.0, r_hi=2.0, seed=BASE_SEED + 1),
    "d5_N1024_k1000": Workload("d5_N1024_k1000", 5, 1024, 1000, (3, 2), seed=BASE_SEED + 2),
    # noisy: a prime floor keeps the read-out noise N sigma / (2 pi sqrt(p) |a|) of |a| = 1 modes
    # four standard deviations inside delta = 0.25
    "d10_N65536_k10000_noisy": Workload("d10_N65536_k10000_noisy", 10, 1 << 16, 10000, (2,) * 5,
                                        noise_sigma=1e-3, seed=BASE_SEED + 3, p_min=30000),
    "d20_N1048576_k100000": Workload("d20_N1048576_k100000", 20, 1 << 20, 100000, (2,) * 10,
                                     r_dist="loguniform", r_lo=1e-2, r_hi=1e2, seed=BASE_SEED + 5),
}


def default_blocks(d: int, N: int, k: int, c: int = 5) -> tuple:
    """Block sizes for partial unwrapping (Sec. 4.1): the smallest b with N^b >= 4 c k,
    d // b blocks, sizes as even as possible (earlier blocks take the remainder)."""
    b = 1
    while N ** b < 4 * c * max(k, 1) and b < d:
        b += 1
    nb = max(1, d // b)
    base, rem = divmod(d, nb)
    return tuple(base + (1 if q < rem else 0) for q in range(nb))


def wide_blocks(d: int, N: int) -> tuple:
    """Block sizes for partial unwrapping (Sec. 4.1) with the widest blocks whose direction
    (N^r on a block's r-th coordinate, Eq. 35) stays an int64: b - 1 = the largest r with
    N^r <= 9e18, ceil(d / b) blocks, sizes as even as possible.  With one shifted set per
    coordinate the read-out resolves N values from one phase whatever the block, so wide blocks
    cost no precision; they give fewer line directions and larger projected ranges."""
    r = 0
    while r + 1 < d and float(N) ** (r + 1) <= 9.0e18:
        r += 1
    b = r + 1
    nb = -(-d // b)
    base, rem = divmod(d, nb)
    return tuple(base + (1 if q < rem else 0) for q in range(nb))


def blocks_for(d: int, N: int, k: int, rule: str = "narrow") -> tuple:
    """Blocks by the named rule: "narrow" (default_blocks) or "wide" (wide_blocks)."""
    if rule == "wide":
        return wide_blocks(d, N)
    if rule == "narrow":
        return default_blocks(d, N, k)
    raise ValueError(rule)


def batched_mix(n_signals: int = 4096, seed: int = BASE_SEED + 4, k_lo: int = 8, k_hi: int = 512,
                d_lo: int = 2, d_hi: int = 8, logN_lo: int = 10, logN_hi: int = 20) -> list:
    """Independent signals with k ~ U{k_lo..k_hi}, d ~ U{d_lo..d_hi}, N = 2^U{logN_lo..logN_hi},
    r ~ U[1, 10], noiseless (the batched workload)."""
    st = Stream(seed)
    ks = st.integers(n_signals, k_lo, k_hi + 1)
    ds = st.integers(n_signals, d_lo, d_hi + 1)
    ls = st.integers(n_signals, logN_lo, logN_hi + 1)
    out = []
    for s in range(n_signals):
        d, N, k = int(ds[s]), 1 << int(ls[s]), int(ks[s])
        sig = draw_signal(d, N, k, seed * 1000003 + s, "uniform", 1.0, 10.0)
        out.append((sig, default_blocks(d, N, k)))
    return out
