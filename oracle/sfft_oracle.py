"""Plain FP64 CPU oracle of the multidimensional phase-shift sparse FFT
(Choi, Christlieb, Wang, "High-Dimensional Sparse Fourier Algorithms").

TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
that the CUDA path is checked against.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library never does.  It
shares no code with the CUDA path: its only common input is the seeded signal
generator, which holds none of the method's arithmetic.

What it computes (Algorithm 2, MultiPhaseshift, in its general form):

  round i = 1, 2, ...:
    k* = max(k - |R|, 1); p = the i-th prime >= c k*             (Alg. 2, prime choice)
    u  = line direction of round i: the partial-unwrap vector of  (Sec. 4.1, Eq. 35-38)
         block m = i mod B, u_l = N^r on the block's r-th digit
    y_n[x] = (f - g)(x u / p + s_n), x = 0..p-1, n = 0..d,        (Alg. 2 sampling; Eq. 41)
         s_0 = 0, s_n = e_n / N  (one shifted copy per coordinate)
    Y_n = DFT_p(y_n)                                             (Eq. 3)
    for every bin h with |Y_0[h]| above the empty-bin level:
         accept iff | |Y_n[h]| / |Y_0[h]| - 1 | < tau for all n   (Eq. 8, Eq. 42)
         w_n = N Arg(Y_n[h] / Y_0[h]) / (2 pi), rounded            (Eq. 7, Eq. 41 with eps = 1/N)
         a   = Y_0[h] / p                                         (Eq. 7, Eq. 41)
    R <- R merged with the accepted (w, a); prune small |a|       (Alg. 2 registry update)
  until empty_rounds rounds in a row (successive line directions; by default one per
  direction) find no bin of any set above the empty-bin level (the residual is empty).

Readings of the paper taken here (each is listed with its reason in the design
notes): per-coordinate shifts e_n / N instead of eps times a block vector; the
box [0, N)^d by default (the paper's [-N/2, N/2)^d via box_lo = -N/2); every
occupied bin is examined instead of the k* largest after a sort; the ratio
tolerance tau is its own parameter; an accepted vector must land in its own bin
((w . u) mod p == h) and round to within delta of an integer; a duplicate key
adds its coefficient to the registry entry; the empty-bin level is rho p A_ref
with A_ref the largest first-round bin divided by p, plus 6 sigma sqrt(p) when
the samples carry noise.

Also here: the block shifts of Alg. 2 as printed (shift "block"), the tilted
lines of Alg. 3 in two dimensions (shift "tilt": rotated axes, rotated shifts,
read-out turned back, Sec. 3.3 and Theorem 1), Alg. 1 in one dimension, and the
worst case of the parallel projections (projection_core: the modes no axis line
ever isolates; worst_case_bound: Sec. 4.2's bound on its probability).

Arithmetic is float64 / complex128 throughout; integer phase indices are
reduced exactly in int64 before any floating point is applied.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
import math

import numpy as np

# --------------------------------------------------------------------------
# Prime schedule (Alg. 1 and Alg. 2: "p <- i-th prime number >= c k*"; c = 5, Sec. 5)
# --------------------------------------------------------------------------


def is_prime(n: int) -> bool:
    """Trial division."""
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    f = 3
    while f * f <= n:
        if n % f == 0:
            return False
        f += 2
    return True


def ith_prime_at_least(i: int, lo: int) -> int:
    """The i-th smallest prime that is >= lo (i >= 1)."""
    if i < 1:
        raise ValueError("i >= 1")
    n, count = max(lo, 2), 0
    while True:
        if is_prime(n):
            count += 1
            if count == i:
                return n
        n += 1


# --------------------------------------------------------------------------
# Line directions: partial unwrapping (Sec. 4.1, Eq. 35-38)
# --------------------------------------------------------------------------


def block_starts(blocks) -> list:
    starts, s = [], 0
    for b in blocks:
        starts.append(s)
        s += b
    return starts


def unwrap_vector(d: int, N: int, blocks, m: int) -> np.ndarray:
    """u with u_l = N^r for coordinate l = (start of block m) + r, r = 0..d_m - 1, else 0.

    Along t = x u / p the phase of mode w is x * (sum_r N^r w_{start+r}) / p, i.e. the
    block-m coordinates unwrapped to one integer (Eq. 35) and sampled at rate 1/p."""
    if sum(blocks) != d:
        raise ValueError("block sizes must add up to d")
    u = np.zeros(d, dtype=object)
    s = block_starts(blocks)[m]
    for r in range(blocks[m]):
        u[s + r] = N ** r
    return u


def line_direction(d: int, N: int, blocks, i: int, dirs=None) -> np.ndarray:
    """Direction of round i (1-based).  With blocks: block m = i mod B (0-based), which is
    the paper's m <- (i mod d2) + 1 in 1-based numbering.  An explicit list of integer
    directions (tilted lines) is used in the same rotation."""
    if dirs is not None and len(dirs) > 0:
        return np.array(dirs[i % len(dirs)], dtype=object)
    return unwrap_vector(d, N, blocks, i % len(blocks))


# --------------------------------------------------------------------------
# Tilted lines in two dimensions (Sec. 3.3, Eq. 21-27, Alg. 3, Theorem 1)
# --------------------------------------------------------------------------


def tilt_axes(tilt) -> np.ndarray:
    """The rotated axes of Alg. 3 in the original coordinates.  With sin = height / hypo and
    cos = base / hypo (Eq. 25), g^(t~) = f(t~_1 base + t~_2 height, -t~_1 height + t~_2 base)
    (Eq. 27 after the factor hypo), so t~ = e_1 is the point (base, -height) and t~ = e_2 the
    point (height, base); a mode w is seen with the rotated frequency
    w~ = (base w_1 - height w_2, height w_1 + base w_2) (Eq. 21 times hypo).
    Row m - 1 is axis m; round i samples along axis (i mod 2) + 1 (Alg. 3), which line_direction
    picks from these rows as dirs[i mod 2]."""
    base, height, _ = (int(v) for v in tilt)
    return np.array([[base, -height], [height, base]], dtype=np.int64)


def tilt_window(N: int, box_lo: int, tilt):
    """(Q, lo): the read-out modulus and the lowest value of each rotated coordinate over the box
    [box_lo, box_lo + N)^2.  Both rotated coordinates span (base + height)(N - 1) + 1 values, so
    the shift eps = 1 / Q with Q = (base + height) N keeps each one unambiguous modulo Q (the
    role of eps in Alg. 3, which leaves its value open)."""
    base, height, _ = (int(v) for v in tilt)
    Q = (base + height) * N
    lo = (base * box_lo - height * (box_lo + N - 1), (base + height) * box_lo)
    return Q, lo


def check_tilt(tilt) -> None:
    """Theorem 1's conditions that the read-out relies on: a Pythagorean triple
    base^2 + height^2 = hypo^2 with gcd(base, height) = 1 (Eq. 25), both legs positive."""
    base, height, hypo = (int(v) for v in tilt)
    if base < 1 or height < 1 or base * base + height * height != hypo * hypo or math.gcd(base, height) != 1:
        raise ValueError("tilt must be a primitive Pythagorean triple (base, height, hypo)")


# --------------------------------------------------------------------------
# Sampling of f - g along the line and its shifted copies (Alg. 2 sampling lines, Eq. 41)
# --------------------------------------------------------------------------


def shift_phases(freqs: np.ndarray, N: int, shift: str = "coord", blocks=None, tilt=None):
    """Exact phases of the shifted sets: (num, q) with w_j . s_n = num[j, n] / q[n] mod 1.

    shift "coord" (the general form): s_n = e_n / N, so the phase of set n is w_n mod N over N.
    shift "block" (Alg. 2 as printed, reading A5): set n moves along the unwrap vector v_n of
    block n (N^r on its r-th coordinate, Eq. 35) by eps_n = 1 / (2 N^{d1_n}), d1_n its size, so
    the phase is w~_n / (2 N^{d1_n}) with w~_n = sum_r w_{b_n + r} N^r the block's unwrapped
    frequency (Eq. 35-36).
    shift "tilt" (Alg. 3, d = 2): set n moves by eps along rotated axis n (tilt_axes), eps = 1 / Q
    (tilt_window), so the phase is w~_n / Q with w~_n the n-th rotated frequency (Eq. 27)."""
    freqs = np.asarray(freqs, dtype=np.int64)
    K, d = freqs.shape
    if shift == "coord":
        return np.mod(freqs, N), np.full(d, N, dtype=np.int64)
    if shift == "tilt":
        Q, _ = tilt_window(N, 0, tilt)
        wt = freqs @ tilt_axes(tilt).T                 # [K, 2]: w . (axis n), exact in int64
        return np.mod(wt, Q), np.full(2, Q, dtype=np.int64)
    starts = block_starts(blocks)
    num = np.zeros((K, len(blocks)), dtype=np.int64)
    q = np.zeros(len(blocks), dtype=np.int64)
    for n, (b, size) in enumerate(zip(starts, blocks)):
        wt = np.zeros(K, dtype=np.int64)
        for r in range(size):
            wt += freqs[:, b + r] * N ** r
        q[n] = 2 * N ** size
        num[:, n] = np.mod(wt, q[n])
    return num, q


def sample_sets(freqs: np.ndarray, coeffs: np.ndarray, p: int, u, N: int,
                chunk: int = 4096, x_values=None, shift: str = "coord", blocks=None,
                tilt=None) -> np.ndarray:
    """y[n, x] = sum_j coeffs_j exp(2 pi i w_j . t_{n,x}),  t_{n,x} = x u / p + s_n,
    s_0 = 0 and s_n = e_n / N, for x = 0..p-1 and n = 0..d.

    f is 1-periodic in every coordinate, so only w . t mod 1 matters.  It is reduced
    exactly: w . (x u / p) = x (w . u) / p, whose fractional part is ((x (w . u)) mod p) / p,
    and w . s_n = w_n / N, whose fractional part is (w_n mod N) / N.  Registry modes enter
    with negated coefficients, so the same call evaluates f - g.  ``x_values``, if given,
    restricts the evaluation to those sample indices (columns in the given order).  With
    shift "block" or "tilt" the shifted sets are those of shift_phases (one per block, or one per
    rotated axis)."""
    freqs = np.asarray(freqs, dtype=np.int64)
    coeffs = np.asarray(coeffs, dtype=np.complex128)
    K, d = freqs.shape
    S = len(blocks) if shift == "block" else d
    xs = np.arange(p, dtype=np.int64) if x_values is None else np.asarray(x_values, dtype=np.int64)
    y = np.zeros((S + 1, xs.size), dtype=np.complex128)
    if K == 0:
        return y
    u_mod = np.array([int(v) % p for v in u], dtype=np.int64)
    alpha = (freqs @ u_mod) % p                       # (w . u) mod p, exact
    num, q = shift_phases(freqs, N, shift, blocks, tilt)
    shift_frac = num / q[None, :]                     # frac(w . s_n) for n = 1..S
    for x0 in range(0, xs.size, chunk):
        x = xs[x0:x0 + chunk]
        line_frac = ((alpha[:, None] * x[None, :]) % p) / p
        for n in range(S + 1):
            frac = line_frac if n == 0 else line_frac + shift_frac[:, n - 1][:, None]
            y[n, x0:x0 + x.size] = coeffs @ np.exp(2j * np.pi * frac)
    return y


def registry_bins(freqs: np.ndarray, coeffs: np.ndarray, p: int, u, N: int, shift: str = "coord",
                  blocks=None, tilt=None) -> np.ndarray:
    """The DFT of the samples of g = sum_j coeffs_j e^{2 pi i w_j . t}, written without sampling:
    sample set n of one mode is a_j e^{2 pi i w_{j,n} / N} W^{alpha_j x} with alpha_j = (w_j . u)
    mod p (see sample_sets), and sum_x W^{(alpha_j - h) x} is p when h = alpha_j and 0 otherwise
    (the DFT of Sec. 2.1), so G[n, h] = p sum_{j : alpha_j = h} a_j e^{2 pi i w_{j,n} / N}
    (the factor is 1 for n = 0).  Removing g from the transform instead of from the samples
    is the adaptive step of Alg. 2 (Sec. 5, "Algorithm") by the linearity of the DFT."""
    freqs = np.asarray(freqs, dtype=np.int64)
    coeffs = np.asarray(coeffs, dtype=np.complex128)
    K, d = freqs.shape
    S = len(blocks) if shift == "block" else d
    G = np.zeros((S + 1, p), dtype=np.complex128)
    if K == 0:
        return G
    u_mod = np.array([int(v) % p for v in u], dtype=np.int64)
    alpha = (freqs @ u_mod) % p
    num, q = shift_phases(freqs, N, shift, blocks, tilt)
    for j in range(K):
        G[0, alpha[j]] += p * coeffs[j]
        for n in range(1, S + 1):
            G[n, alpha[j]] += p * coeffs[j] * np.exp(2j * np.pi * int(num[j, n - 1]) / int(q[n - 1]))
    return G


def dft(y: np.ndarray) -> np.ndarray:
    """Y[h] = sum_x y[x] exp(-2 pi i h x / p) along the last axis (the DFT defined in Sec. 2.1)."""
    return np.fft.fft(y, axis=-1)


# --------------------------------------------------------------------------
# Noise of the black box: the Philox4x32-10 counter-based generator
# --------------------------------------------------------------------------

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57   # round multipliers
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85   # key increments between rounds
_M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
    as 1, 2, 3", SC 2011), vectorised over arrays of 32-bit values.  One round multiplies c0 by
    M0 and c2 by M1 into 64-bit products (hi, lo) and sets
        c <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key (k0, k1) advances by the two increments between rounds."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _M32 for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & _M32
            k1 = (k1 + np.uint64(_PHILOX_W1)) & _M32
        p0 = c0 * np.uint64(_PHILOX_M0)   # < 2^64: exact in uint64
        p1 = c2 * np.uint64(_PHILOX_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def black_box_noise(seed: int, round_i: int, p: int, d: int, sigma: float) -> np.ndarray:
    """Noise added to the black box's samples of round i (complex [d + 1, p]), Re and Im each
    N(0, sigma^2 / 2).  Sample (set n, point x) takes Philox4x32-10 of the counter
    (x, n, i, 0) under the key (seed mod 2^32, seed div 2^32); its first two words give
    u1 = (w0 + 1/2) / 2^32 in (0, 1) and u2 = w1 / 2^32, and the Box-Muller transform gives
    sqrt(-2 ln u1) e^{2 pi i u2} sigma / sqrt(2)."""
    x = np.tile(np.arange(p, dtype=np.uint64), d + 1)
    n = np.repeat(np.arange(d + 1, dtype=np.uint64), p)
    w0, w1, _, _ = philox4x32_10(x, n, np.full(x.shape, round_i, dtype=np.uint64), np.zeros_like(x),
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = (w0.astype(np.float64) + 0.5) / 2.0 ** 32
    u2 = w1.astype(np.float64) / 2.0 ** 32
    z = np.sqrt(-2.0 * np.log(u1)) * np.exp(2j * np.pi * u2) * (sigma / math.sqrt(2.0))
    return z.reshape(d + 1, p)


# --------------------------------------------------------------------------
# Bin test, frequency and coefficient read-out (Eq. 7-8, Eq. 41-42)
# --------------------------------------------------------------------------


def arg(z: np.ndarray) -> np.ndarray:
    """Arg in [-pi, pi) (Sec. 2.1)."""
    a = np.angle(z)
    return np.where(a >= np.pi, a - 2 * np.pi, a)


@dataclass
class Thresholds:
    tau: float = 1e-7        # ratio-test tolerance (Eq. 8, Eq. 42)
    rho: float = 2.0 ** -40  # empty-bin level relative to the first round's largest bin
    delta: float = 0.1       # largest distance of N Arg / (2 pi) from an integer
    sigma: float = 0.0       # noise level of the samples (adds 6 sigma sqrt(p) to the level)


def _decode_blocks(ratio: np.ndarray, N: int, blocks, box_lo: int, delta: float, d: int):
    """Frequency vector from the block read-outs, or None when a read-out is farther than delta
    from an integer or falls outside the box's window of unwrapped values."""
    w = np.zeros(d, dtype=np.int64)
    for n, (b, size) in enumerate(zip(block_starts(blocks), blocks)):
        q = 2 * N ** size
        v = q * float(arg(ratio[n])) / (2 * np.pi)
        r = round(v)
        if abs(v - r) > delta:
            return None
        lo = box_lo * sum(N ** t for t in range(size))              # unwrapped value of (box_lo, ...)
        t = (r - lo) % q
        if t >= N ** size:
            return None
        for pos in range(size):                                      # base-N digits, lowest first
            w[b + pos] = t % N + box_lo
            t //= N
    return w


def _decode_tilt(ratio: np.ndarray, N: int, tilt, box_lo: int, delta: float):
    """Frequency pair from the two rotated read-outs (Alg. 3), or None.  Set n gives
    w~_n = Q Arg(Y_n / Y_0) / (2 pi) (eps = 1 / Q), taken in the window of the box's rotated
    values; the pair is turned back with [cos sin; -sin cos] (Alg. 3, last step).  The rotated
    frequencies carry the factor hypo (Eq. 27), so the turn gives hypo^2 w: a pair that is not
    an exact multiple of hypo^2, or lands outside the box, is no mode's read-out and is
    rejected."""
    base, height, hypo = (int(v) for v in tilt)
    Q, lo = tilt_window(N, box_lo, tilt)
    wt = []
    for n in range(2):
        v = Q * float(arg(ratio[n])) / (2 * np.pi)
        r = round(v)
        if abs(v - r) > delta:
            return None
        wt.append(lo[n] + (r - lo[n]) % Q)
    c2 = hypo * hypo
    x1 = base * wt[0] + height * wt[1]
    x2 = -height * wt[0] + base * wt[1]
    if x1 % c2 or x2 % c2:
        return None
    w = np.array([x1 // c2, x2 // c2], dtype=np.int64)
    if np.any(w < box_lo) or np.any(w >= box_lo + N):
        return None
    return w


def classify(Y: np.ndarray, p: int, u, N: int, eta_bin: float, th: Thresholds,
             box_lo: int = 0, estimator: str = "set0", shift: str = "coord", blocks=None, tilt=None):
    """All bins h = 0..p-1 that hold exactly one mode, with the mode read off.

    The coefficient is a = Y_0[h] / p (Eq. 41, estimator "set0") or, with estimator
    "mean", the mean over n = 0..d of Y_n[h] exp(-2 pi i w_n / N) / p, which for a bin
    holding one mode has every term equal to a (Eq. 41 applied to each shifted set).
    Returns a list of (h, w, a), w a tuple of d ints, in increasing h.

    With shift "block" set n reads the unwrapped frequency of block n,
    w~_n = 2 N^{d1} Arg(Y_n / Y_0) / (2 pi) (Alg. 2 read-out with eps = 1 / (2 N^{d1})), taken in
    the window of the box's unwrapped values and split into its d1 base-N digits (Alg. 2 wrap-back).
    With shift "tilt" the two sets read the rotated pair, turned back by _decode_tilt (Alg. 3)."""
    Y0 = Y[0]
    occupied = np.abs(Y0) > eta_bin
    out = []
    u_mod = np.array([int(v) % p for v in u], dtype=np.int64)
    d = len(u_mod)
    for h in np.nonzero(occupied)[0]:
        ratio = np.abs(Y[1:, h]) / np.abs(Y0[h])                    # Eq. 42, every n
        if not np.all(np.abs(ratio - 1.0) < th.tau):
            continue
        if shift == "coord":
            v = N * arg(Y[1:, h] / Y0[h]) / (2 * np.pi)             # Eq. 41 with eps = 1/N
            r = np.round(v)
            if not np.all(np.abs(v - r) <= th.delta):
                continue
            w = (np.mod(r.astype(np.int64) - box_lo, N) + box_lo).astype(np.int64)
        elif shift == "tilt":
            w = _decode_tilt(Y[1:, h] / Y0[h], N, tilt, box_lo, th.delta)
            if w is None:
                continue
        else:
            w = _decode_blocks(Y[1:, h] / Y0[h], N, blocks, box_lo, th.delta, d)
            if w is None:
                continue
        if int(w @ u_mod) % p != h:                                  # lands in its own bin
            continue
        if estimator == "mean":
            num, q = shift_phases(w[None, :], N, shift, blocks, tilt)
            rot = np.concatenate([[1.0 + 0j], np.exp(-2j * np.pi * num[0] / q)])
            a = complex(np.mean(Y[:, h] * rot) / p)
        else:
            a = complex(Y0[h] / p)                                   # Eq. 41: a = Y_0 / p
        out.append((int(h), tuple(int(c) for c in w), a))
    return out


# --------------------------------------------------------------------------
# Worst case of the parallel projections (Sec. 2.2, Sec. 4.2)
# --------------------------------------------------------------------------


def unwrapped_coordinates(freqs: np.ndarray, N: int, blocks, box_lo: int = 0) -> np.ndarray:
    """[K, B] the block-unwrapped coordinates w~_q = sum_r (w_{b_q + r} - box_lo) N^r (Eq. 35),
    the values the line of block q separates the modes by (Python ints: N^{d1} may pass 2^63)."""
    freqs = np.asarray(freqs, dtype=np.int64)
    out = np.empty((freqs.shape[0], len(blocks)), dtype=object)
    for q, (b, size) in enumerate(zip(block_starts(blocks), blocks)):
        for j in range(freqs.shape[0]):
            out[j, q] = sum((int(freqs[j, b + r]) - box_lo) * N ** r for r in range(size))
    return out


def projection_core(freqs: np.ndarray, N: int, blocks, box_lo: int = 0) -> np.ndarray:
    """Indices of the modes that the parallel projections never isolate (the worst case of
    Sec. 2.2 and 3.3): two modes with the same unwrapped coordinate q share a bin on every line of
    block q whatever the prime, while modes whose coordinates differ are apart for all but the
    primes dividing the difference.  A mode whose coordinate q no other remaining mode shares is
    found on block q's lines and leaves the residual; removing those repeatedly leaves the modes
    that every projection keeps in a bin with another (the rectangle corners of two dimensions)."""
    wt = unwrapped_coordinates(freqs, N, blocks, box_lo)
    alive = set(range(wt.shape[0]))
    changed = True
    while changed:
        changed = False
        for q in range(wt.shape[1]):
            count: dict = {}
            for j in alive:
                count[wt[j, q]] = count.get(wt[j, q], 0) + 1
            lone = {j for j in alive if count[wt[j, q]] == 1}
            if lone:
                alive -= lone
                changed = True
    return np.array(sorted(alive), dtype=np.int64)


def worst_case_bound(N: int, blocks, k: int) -> float:
    """Sec. 4.2's upper bound on the probability that the parallel projections fail for k modes
    drawn uniformly from N^d vectors with the blocks' unwrapping: 1 - prod_{j=1..k} P(A_j), where
    A_j is the j-th vector avoiding the axis-parallel lines (in the unwrapped coordinates) through
    the earlier ones, P(A_j) >= (N^d - (j - 1) sum_q N^{d_q}) / N^d.  Evaluated exactly, clipped
    at 1."""
    from fractions import Fraction
    d = sum(blocks)
    total = N ** d
    line = sum(N ** b for b in blocks)
    prod = Fraction(1)
    for j in range(1, k + 1):
        f = Fraction(total - (j - 1) * line, total)
        if f <= 0:
            return 1.0
        prod *= f
    return float(1 - prod)


# --------------------------------------------------------------------------
# Algorithm 2 driver
# --------------------------------------------------------------------------


@dataclass
class Result:
    freqs: np.ndarray            # int64 [n, d], lexicographically sorted
    coeffs: np.ndarray           # complex128 [n]
    converged: bool
    rounds: list = field(default_factory=list)   # per-round dicts

    @property
    def n_found(self) -> int:
        return int(self.freqs.shape[0])

    @property
    def samples(self) -> int:
        return int(sum(r["samples"] for r in self.rounds))


def multi_phaseshift(freqs, coeffs, d: int, N: int, k: int, blocks=None, c: float = 5,
                     th: Thresholds | None = None, max_rounds: int | None = None,
                     box_lo: int = 0, primes=None, dirs=None, noise=None,
                     estimator: str = "set0", residual: str = "samples", p_min: int = 0,
                     shift: str = "coord", tilt=None, empty_rounds: int | None = None) -> Result:
    """Algorithm 2 (MultiPhaseshift) on the black box f = sum_j coeffs_j e^{2 pi i freqs_j . t}.

    ``primes``, if given, overrides the prime rule (round i uses primes[(i-1) mod len]).
    ``noise``, if given, is a callable (i, p, d) -> complex array [d+1, p] added to the
    black-box samples of round i.  ``residual`` says where g (built from the registry) leaves
    f: "samples" evaluates f - g at every sample point, as Alg. 2 writes it; "bins" samples f
    alone and subtracts the transform of g bin by bin (registry_bins).  ``p_min`` floors the
    prime rule: round i uses the i-th prime >= max(c k*, p_min).  ``shift`` is "coord" (one
    shifted set per coordinate, s_n = e_n / N), "block" (one per block, Alg. 2 as printed) or
    "tilt" (d = 2, Alg. 3: ``tilt`` = (base, height, hypo); the lines run along the rotated axes
    in turn unless ``dirs`` is given, and the sets shift along them).  ``empty_rounds`` rounds in a
    row with no bin of any set above the empty-bin level end the run (default: the number of line
    directions)."""
    if residual not in ("samples", "bins"):
        raise ValueError(residual)
    if shift == "tilt":
        if d != 2:
            raise ValueError("the tilted form (Alg. 3) is two-dimensional")
        check_tilt(tilt)
        if dirs is None:
            dirs = [tuple(int(v) for v in row) for row in tilt_axes(tilt)]
    th = th or Thresholds()
    freqs = np.asarray(freqs, dtype=np.int64).reshape(-1, d)
    coeffs = np.asarray(coeffs, dtype=np.complex128).reshape(-1)
    if blocks is None:
        blocks = (d,)
    if max_rounds is None:
        max_rounds = 64 + 4 * max(1, math.ceil(math.log2(max(k, 2))))
    R: dict = {}                       # registry: w -> a, in insertion order
    a_ref = None
    n_dirs = len(dirs) if dirs is not None and len(dirs) > 0 else len(blocks)
    if empty_rounds is None:
        empty_rounds = n_dirs
    empty_streak = 0
    rounds = []
    converged = False
    for i in range(1, max_rounds + 1):
        k_star = max(k - len(R), 1)
        # "p <- i-th prime >= c k*": the smallest integer at or above c k* is ceil(c k*), taken
        # exactly (c may be a fraction such as 5/2; Alg. 2 leaves c to the caller)
        p = (int(primes[(i - 1) % len(primes)]) if primes is not None
             else ith_prime_at_least(i, max(math.ceil(Fraction(c) * k_star), p_min)))
        u = line_direction(d, N, blocks, i, dirs)
        # f - g: black-box modes with +a, registry modes with -a (Alg. 2: g is built from R)
        if R and residual == "samples":
            reg_w = np.array(list(R.keys()), dtype=np.int64).reshape(-1, d)
            reg_a = -np.array(list(R.values()), dtype=np.complex128)
            all_w = np.concatenate([freqs, reg_w])
            all_a = np.concatenate([coeffs, reg_a])
        else:
            all_w, all_a = freqs, coeffs
        y = sample_sets(all_w, all_a, p, u, N, shift=shift, blocks=blocks, tilt=tilt)
        if noise is not None:
            y = y + noise(i, p, y.shape[0] - 1)
        Y = dft(y)
        if R and residual == "bins":
            reg_w = np.array(list(R.keys()), dtype=np.int64).reshape(-1, d)
            Y = Y - registry_bins(reg_w, np.array(list(R.values()), dtype=np.complex128), p, u, N,
                                  shift=shift, blocks=blocks, tilt=tilt)
        if a_ref is None:
            a_ref = float(np.max(np.abs(Y[0]))) / p if p > 0 else 0.0
        eta_bin = max(th.rho * p * a_ref, 6.0 * th.sigma * math.sqrt(p))
        stat = {"round": i, "p": p, "k_star": k_star, "terms": int(all_w.shape[0]),
                "samples": int(Y.shape[0]) * p, "eta_bin": eta_bin}
        # the residual is empty when no bin of any set is above the level, in empty_rounds rounds
        # in a row (successive line directions): a registry pair of opposite coefficients that a
        # line does not separate cancels in set 0, and when the pair differs by a few units in
        # one coordinate its shifted sets differ by a phase of only 2 pi (w_n - w'_n) / N; a line
        # of the block where they differ, with another prime, puts the two in different bins
        if not np.any(np.abs(Y) > eta_bin):
            empty_streak += 1
            stat.update(accepted=0, registry=len(R))
            rounds.append(stat)
            if empty_streak >= empty_rounds:
                converged = True
                break
            continue
        empty_streak = 0
        acc = classify(Y, p, u, N, eta_bin, th, box_lo, estimator, shift=shift, blocks=blocks, tilt=tilt)
        for _, w, a in acc:                                    # R <- R u (w, a)
            R[w] = R.get(w, 0j) + a
        eta_prune = max(th.rho * a_ref, 6.0 * th.sigma / math.sqrt(p))
        for w in [w for w, a in R.items() if abs(a) < eta_prune]:   # prune small coefficients
            del R[w]
        stat.update(accepted=len(acc), registry=len(R))
        rounds.append(stat)
    keys = sorted(R.keys())
    out_w = np.array(keys, dtype=np.int64).reshape(-1, d)
    out_a = np.array([R[w] for w in keys], dtype=np.complex128)
    return Result(out_w, out_a, converged, rounds)


# --------------------------------------------------------------------------
# Algorithm 1 (one-dimensional Phaseshift), kept literal as a special-case check
# --------------------------------------------------------------------------


def phaseshift_1d(freqs, coeffs, N: int, k: int, c: int = 5, tau: float = 1e-7,
                  max_rounds: int = 200, rho: float = 2.0 ** -40):
    """Alg. 1 with eps = 1/N: samples f - g at h/p and h/p + eps, FFTs both, sorts the
    unshifted transform by magnitude, tests the k* largest bins, reads w and a (Eq. 7),
    merges into R, prunes, repeats while |R| < k.  Frequencies are taken in [0, N)."""
    freqs = np.asarray(freqs, dtype=np.int64).reshape(-1)
    coeffs = np.asarray(coeffs, dtype=np.complex128).reshape(-1)
    R: dict = {}
    a_ref = None
    for i in range(1, max_rounds + 1):
        if len(R) >= k:
            break
        k_star = k - len(R)
        p = ith_prime_at_least(i, c * k_star)
        ws = np.array(list(freqs) + list(R.keys()), dtype=np.int64)
        as_ = np.array(list(coeffs) + [-a for a in R.values()], dtype=np.complex128)
        x = np.arange(p)
        t0 = x / p
        f0 = np.array([np.sum(as_ * np.exp(2j * np.pi * ws * t)) for t in t0])
        fe = np.array([np.sum(as_ * np.exp(2j * np.pi * ws * (t + 1.0 / N))) for t in t0])
        F0, Fe = np.fft.fft(f0), np.fft.fft(fe)
        if a_ref is None:
            a_ref = np.max(np.abs(F0)) / p
        order = np.argsort(-np.abs(F0), kind="stable")             # SORT by |F_0|
        for h in order[:k_star]:
            if np.abs(F0[h]) <= rho * p * a_ref:
                continue
            if abs(np.abs(Fe[h]) / np.abs(F0[h]) - 1.0) < tau:      # Eq. 8
                w = int(np.round(N * arg(Fe[h] / F0[h]) / (2 * np.pi))) % N   # Eq. 7
                R[w] = R.get(w, 0j) + F0[h] / p
        for w in [w for w, a in R.items() if abs(a) < rho * a_ref]:
            del R[w]
    keys = sorted(R.keys())
    return np.array(keys, dtype=np.int64), np.array([R[w] for w in keys], dtype=np.complex128)


# --------------------------------------------------------------------------
# Brute-force checker: full d-dimensional DFT of the black box on its grid
# --------------------------------------------------------------------------


def full_grid_coefficients(freqs, coeffs, d: int, N: int, box_lo: int = 0) -> np.ndarray:
    """Samples f on the grid t = g / N, g in [0, N)^d, and returns the d-dimensional DFT
    divided by N^d: entry (w - box_lo) mod N holds the coefficient of frequency w.
    Only for N^d small enough to hold in memory."""
    freqs = np.asarray(freqs, dtype=np.int64).reshape(-1, d)
    coeffs = np.asarray(coeffs, dtype=np.complex128)
    grids = np.meshgrid(*[np.arange(N)] * d, indexing="ij")
    f = np.zeros([N] * d, dtype=np.complex128)
    for w, a in zip(freqs, coeffs):
        ph = sum(int(w[l]) * grids[l] for l in range(d)) % N
        f += a * np.exp(2j * np.pi * ph / N)
    F = np.fft.fftn(f) / N ** d
    # fftn uses e^{-2 pi i g.v/N}: the coefficient of w sits at index v = w mod N
    if box_lo != 0:
        F = np.roll(F, shift=[-box_lo] * d, axis=tuple(range(d)))
    return F
