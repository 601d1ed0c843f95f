"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each check ties one step of the oracle to something the paper or mathematics fixes:
printed worked examples (tests/golden), closed forms, brute force on tiny inputs,
a textbook routine (the full d-dimensional FFT), and invariants (Parseval).
``test_planted_mistakes_are_caught`` plants plausible slips in the oracle and
shows that these checks notice each one.
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import oracle.sfft_oracle as O
from paper_1606_07407_gb300.inputs import draw_signal, Stream

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def _sieve(n):
    s = np.ones(n + 1, dtype=bool)
    s[:2] = False
    for q in range(2, int(n ** 0.5) + 1):
        if s[q]:
            s[q * q::q] = False
    return np.nonzero(s)[0]


# ---------------------------------------------------------------- primes

def test_prime_rule_matches_sieve_and_golden():
    pr = _sieve(600000)
    for lo in (2, 5, 80, 997, 5000, 50000, 500000):
        first = np.searchsorted(pr, lo)
        for i in (1, 2, 7):
            assert O.ith_prime_at_least(i, lo) == pr[first + i - 1]
    for row in _rows("primes_first_round.txt"):
        if len(row) == 3 and int(row[1]) == 5 * int(row[0]):
            assert O.ith_prime_at_least(1, int(row[1])) == int(row[2])
        else:
            i, lo, p = map(int, row)
            assert O.ith_prime_at_least(i, lo) == p


# ---------------------------------------------------------------- directions

def test_unwrap_matches_4d_example():
    for N, m, *u in (list(map(int, r)) for r in _rows("unwrap_4d.txt")):
        got = O.unwrap_vector(4, N, (2, 2), m)
        assert [int(v) for v in got] == u


def test_unwrapping_is_injective_on_a_block():
    # Eq. 35 is one-to-one on [0, N)^{d1}: every digit vector gives a distinct integer.
    N, d1 = 5, 3
    u = O.unwrap_vector(d1, N, (d1,), 0)
    vals = {int(np.dot(w, u)) for w in np.ndindex(*([N] * d1))}
    assert len(vals) == N ** d1 and min(vals) == 0 and max(vals) == N ** d1 - 1


# ---------------------------------------------------------------- sampling

def _check_samples_against_rationals(sample_fn):
    rng = Stream(11)
    d, N, p = 3, 8, 7
    freqs = rng.integers(4 * d, 0, N).reshape(4, d)
    coeffs = rng.uniform(4) + 1j * rng.uniform(4)
    u = [1, N, 0]
    y = sample_fn(freqs, coeffs, p, u, N)
    for n in range(d + 1):
        for x in range(p):
            t = [Fraction(x * u[l], p) + (Fraction(1, N) if l == n - 1 else 0) for l in range(d)]
            want = 0j
            for w, a in zip(freqs, coeffs):
                ph = sum(int(w[l]) * t[l] for l in range(d))
                ph -= math.floor(ph)
                want += a * complex(math.cos(2 * math.pi * ph), math.sin(2 * math.pi * ph))
            assert abs(y[n, x] - want) < 1e-12


def test_samples_equal_exact_rational_evaluation():
    _check_samples_against_rationals(O.sample_sets)


def _check_block_samples_against_rationals(sample_fn):
    # Alg. 2 as printed: set n moves along the unwrap vector v_n of block n (N^r on its r-th
    # coordinate) by eps_n = 1 / (2 N^{d1}); exact rational phases, then cos / sin
    rng = Stream(12)
    d, N, p, blocks = 5, 6, 11, (2, 3)
    freqs = rng.integers(4 * d, -3, 3).reshape(4, d)
    coeffs = rng.uniform(4) + 1j * rng.uniform(4)
    u = [1, N, 0, 0, 0]
    y = sample_fn(freqs, coeffs, p, u, N)
    starts = [0, 2]
    assert y.shape == (3, p)
    for n in range(3):
        shift = [Fraction(0)] * d
        if n:
            b, size = starts[n - 1], blocks[n - 1]
            for r in range(size):
                shift[b + r] = Fraction(N ** r, 2 * N ** size)
        for x in range(p):
            t = [Fraction(x * u[l], p) + shift[l] for l in range(d)]
            want = 0j
            for w, a in zip(freqs, coeffs):
                ph = sum(int(w[l]) * t[l] for l in range(d))
                ph -= math.floor(ph)
                want += a * complex(math.cos(2 * math.pi * ph), math.sin(2 * math.pi * ph))
            assert abs(y[n, x] - want) < 1e-12


def test_block_shift_samples_equal_exact_rational_evaluation():
    _check_block_samples_against_rationals(
        lambda f, a, p, u, N: O.sample_sets(f, a, p, u, N, shift="block", blocks=(2, 3)))


def test_block_readout_decodes_every_vector_of_a_box():
    # every vector of the box [-2, 2)^3 (N = 4, one block of 3): its set-1 ratio e^{2 pi i w~ / (2 N^3)}
    # reads back exactly, and a read-out outside the box's window is rejected
    N, blocks, box_lo = 4, (3,), -2
    for w in np.stack(np.meshgrid(*[np.arange(-2, 2)] * 3, indexing="ij"), -1).reshape(-1, 3):
        num, q = O.shift_phases(w[None, :], N, "block", blocks)
        ratio = np.array([np.exp(2j * np.pi * num[0, 0] / q[0])])
        assert np.array_equal(O._decode_blocks(ratio, N, blocks, box_lo, 0.1, 3), w)
    lo = box_lo * (1 + N + N * N)
    outside = np.array([np.exp(2j * np.pi * (lo + N ** 3 + 5) / (2 * N ** 3))])
    assert O._decode_blocks(outside, N, blocks, box_lo, 0.1, 3) is None


# ---------------------------------------------------------------- tilted lines (Sec. 3.3, Alg. 3)

TILT_16 = (40, 9, 41)   # base, height, hypo: 40^2 + 9^2 = 41^2, base > 2 N for N = 16 (Theorem 1)
TILT_32 = (84, 13, 85)  # base > 2 N for N = 32


def _box(N, lo):
    g = np.arange(lo, lo + N)
    return np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)


def test_tilt_theorem1_rotated_coordinates_separate_every_pair_of_the_box():
    # Theorem 1: with tan(theta) = height / base, base > 2N and gcd(base, height) = 1, no two
    # frequency pairs of the box share either rotated coordinate (brute force over all pairs);
    # the triple (4, 3, 5) at the same N breaks the condition and has such pairs
    for N, lo in ((16, 0), (16, -8)):
        W = _box(N, lo)
        for tilt, distinct in ((TILT_16, True), ((4, 3, 5), False)):
            wt = W @ O.tilt_axes(tilt).T
            sep = all(len(set(wt[:, m].tolist())) == len(W) for m in range(2))
            assert sep == distinct


def _check_tilt_samples_against_rationals(sample_fn):
    # Eq. 27: g^(t~) = f(t~_1 base + t~_2 height, -t~_1 height + t~_2 base), sampled at
    # t~ = (x / p) e_m + eps e_n (Alg. 3), eps = 1 / ((base + height) N); exact rational phases
    rng = Stream(21)
    N, p = 16, 13
    base, height, _ = TILT_16
    eps = Fraction(1, (base + height) * N)
    freqs = rng.integers(8, 0, N).reshape(4, 2)
    coeffs = rng.uniform(4) + 1j * rng.uniform(4)
    for m in (1, 2):
        u = [base, -height] if m == 1 else [height, base]
        y = sample_fn(freqs, coeffs, p, u, N)
        assert y.shape == (3, p)
        for n in range(3):
            for x in range(p):
                tt = [Fraction(x, p) if m == 1 else Fraction(0), Fraction(x, p) if m == 2 else Fraction(0)]
                if n:
                    tt[n - 1] += eps
                t = (tt[0] * base + tt[1] * height, -tt[0] * height + tt[1] * base)
                want = 0j
                for w, a in zip(freqs, coeffs):
                    ph = int(w[0]) * t[0] + int(w[1]) * t[1]
                    ph -= math.floor(ph)
                    want += a * complex(math.cos(2 * math.pi * ph), math.sin(2 * math.pi * ph))
                assert abs(y[n, x] - want) < 1e-12


def test_tilt_samples_equal_exact_rational_evaluation():
    _check_tilt_samples_against_rationals(
        lambda f, a, p, u, N: O.sample_sets(f, a, p, u, N, shift="tilt", tilt=TILT_16))


def test_tilt_readout_decodes_every_pair_of_a_box_and_rejects_the_rest():
    # a bin holding one mode has Y_n / Y_0 = e^{2 pi i eps w~_n}, w~ = hypo (w_1 cos - w_2 sin,
    # w_1 sin + w_2 cos) (Eq. 21 times hypo); every pair of the box must read back exactly, and
    # a rotated pair that is no box pair's image must be rejected
    base, height, hypo = TILT_16
    for N, lo in ((16, 0), (16, -8)):
        Q = (base + height) * N
        for w in _box(N, lo):
            wt = (base * int(w[0]) - height * int(w[1]), height * int(w[0]) + base * int(w[1]))
            ratio = np.exp(2j * np.pi * np.array(wt, dtype=float) / Q)
            assert np.array_equal(O._decode_tilt(ratio, N, TILT_16, lo, 0.1), w)
            for dw in ((1, 0), (0, 1), (hypo, 0)):
                bad = np.exp(2j * np.pi * np.array([wt[0] + dw[0], wt[1] + dw[1]], dtype=float) / Q)
                assert O._decode_tilt(bad, N, TILT_16, lo, 0.1) is None


def _rectangles(N):
    # corners of two axis-aligned rectangles: every mode shares its first coordinate with one
    # other mode and its second with another, so every parallel projection collides
    xs, ys, xs2, ys2 = (3, N - 5), (5, N - 3), (8, N - 11), (11, N - 2)
    return np.array([(x, y) for x in xs for y in ys] + [(x, y) for x in xs2 for y in ys2], dtype=np.int64)


def test_tilt_recovers_the_worst_case_that_parallel_projections_cannot():
    # Sec. 3.3: rectangle corners defeat the parallel projections (blocks of 1, lines along e_1
    # and e_2: no mode is ever alone in its bin); Alg. 3's tilted lines recover the planted set
    N = 32
    freqs = _rectangles(N)
    k = len(freqs)
    rng = Stream(22)
    coeffs = (1 + rng.uniform(k)) * np.exp(2j * np.pi * rng.uniform(k))
    o = np.lexsort(freqs.T[::-1])
    par = O.multi_phaseshift(freqs, coeffs, 2, N, k, (1, 1), max_rounds=12, residual="bins")
    assert not par.converged and par.n_found == 0
    for residual in ("samples", "bins"):
        r = O.multi_phaseshift(freqs, coeffs, 2, N, k, shift="tilt", tilt=TILT_32, residual=residual)
        assert r.converged and np.array_equal(r.freqs, freqs[o])
        assert np.max(np.abs(r.coeffs - coeffs[o])) < 1e-13


def test_tilt_recovery_equals_coordinate_shift_recovery():
    # the tilted form reads the same modes as the per-coordinate form, FP64 coefficients at round-off
    for N, k, box, seed in ((32, 24, 0, 23), (64, 60, -32, 24)):
        tilt = TILT_32 if N == 32 else (144, 17, 145)
        sig = draw_signal(2, N, k, seed=seed, box_lo=box)
        o = np.lexsort(sig.freqs.T[::-1])
        rt = O.multi_phaseshift(sig.freqs, sig.coeffs, 2, N, k, box_lo=box, shift="tilt", tilt=tilt,
                                residual="bins")
        rc = O.multi_phaseshift(sig.freqs, sig.coeffs, 2, N, k, (1, 1), box_lo=box, residual="bins")
        assert rt.converged and np.array_equal(rt.freqs, sig.freqs[o].astype(np.int64))
        assert np.array_equal(rt.freqs, rc.freqs)
        assert np.max(np.abs(rt.coeffs - sig.coeffs[o])) < 1e-13


def test_tilt_needs_a_primitive_pythagorean_triple_in_two_dimensions():
    for bad in ((4, 3, 6), (6, 8, 10), (0, 1, 1)):
        with pytest.raises(ValueError):
            O.check_tilt(bad)
    with pytest.raises(ValueError):
        O.multi_phaseshift(np.zeros((1, 3), dtype=np.int64), np.ones(1), 3, 16, 1, shift="tilt", tilt=TILT_16)


# ---------------------------------------------------------------- worst case of the parallel projections (Sec. 4.2)

def test_projection_core_in_two_dimensions_is_the_two_core_of_the_row_column_graph():
    # in two dimensions a mode is an edge between its x value and its y value; a mode with a
    # coordinate no other mode shares hangs off a degree-1 vertex, so peeling leaves exactly the
    # edges of the graph's 2-core (networkx's k_core, a library routine)
    nx = pytest.importorskip("networkx")
    for seed in range(40):
        sig = draw_signal(2, 12, 10 + seed % 20, seed=500 + seed)
        G = nx.Graph()
        G.add_edges_from((("x", int(w[0])), ("y", int(w[1]))) for w in sig.freqs)
        core_nodes = set(nx.k_core(G, 2).nodes)
        want = sorted(j for j, w in enumerate(sig.freqs)
                      if ("x", int(w[0])) in core_nodes and ("y", int(w[1])) in core_nodes)
        assert O.projection_core(sig.freqs, 12, (1, 1)).tolist() == want
    corners = np.array([(1, 2), (1, 7), (5, 2), (5, 7), (9, 9)])
    assert O.projection_core(corners, 12, (1, 1)).tolist() == [0, 1, 2, 3]


def test_parallel_projections_fail_exactly_on_the_projection_core():
    # Alg. 2 with parallel projections leaves out the core's modes and no other, and stops
    # unconverged exactly when the core is not empty (d = 2, blocks of 1; d = 3 with a block of 2)
    n_fail = 0
    for d, N, k, blocks, seeds in ((2, 16, 12, (1, 1), range(40)), (3, 6, 24, (2, 1), range(20))):
        for seed in seeds:
            sig = draw_signal(d, N, k, seed=600 + seed)
            core = set(O.projection_core(sig.freqs, N, blocks).tolist())
            r = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, residual="bins", max_rounds=40)
            found = {tuple(int(v) for v in w) for w in r.freqs}
            missing = {j for j in range(k) if tuple(int(v) for v in sig.freqs[j]) not in found}
            assert missing == core and r.converged == (not core) and r.n_found == k - len(core)
            n_fail += bool(core)
    assert n_fail >= 3   # the cases include failures


def test_worst_case_bound_closed_form_and_monte_carlo():
    # Sec. 4.2: with tau = N^d / sum_q N^{d_q} an integer the product is tau! / ((tau - k)! tau^k);
    # the bound covers the probability of a pair on a common axis-parallel line (event A's
    # complement) and, in two dimensions, the failure probability itself
    for N, blocks, k in ((32, (1, 1), 8), (16, (1, 1), 5), (8, (2, 2), 10)):
        d = sum(blocks)
        tau = N ** d // sum(N ** b for b in blocks)
        exact = 1 - math.factorial(tau) / (math.factorial(tau - k) * tau ** k)
        assert abs(O.worst_case_bound(N, blocks, k) - exact) < 1e-12
    assert O.worst_case_bound(8, (1, 1), 9) == 1.0   # j - 1 >= tau: a factor reaches 0
    N, blocks, k, T = 16, (1, 1), 6, 3000
    pair = fail = 0
    for t in range(T):
        sig = draw_signal(2, N, k, seed=10_000 + t)
        w = sig.freqs
        shared = any(w[i, 0] == w[j, 0] or w[i, 1] == w[j, 1] for i in range(k) for j in range(i))
        pair += shared
        fail += len(O.projection_core(w, N, blocks)) > 0
    bound = O.worst_case_bound(N, blocks, k)
    se = math.sqrt(bound * (1 - bound) / T)
    assert fail <= pair and pair / T < bound + 4 * se


def test_block_shift_recovery_equals_coordinate_shift_recovery():
    # the two shift forms read the same modes (the paper's shape included: d = 100, N = 20,
    # d1 = 5, |a| = 1, signed box) with FP64 coefficients at round-off
    for d, N, k, blocks, box, seed, unit in ((4, 8, 20, (2, 2), 0, 1, False), (6, 16, 40, (3, 3), -8, 2, False),
                                             (100, 20, 16, (5,) * 20, -10, 3, True)):
        sig = draw_signal(d, N, k, seed=seed, box_lo=box, unit_modulus=unit)
        th = O.Thresholds()
        rb = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, th=th, box_lo=box, shift="block")
        rc = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, th=th, box_lo=box)
        o = np.lexsort(sig.freqs.T[::-1])
        assert rb.converged and np.array_equal(rb.freqs, sig.freqs[o].astype(np.int64))
        assert np.array_equal(rb.freqs, rc.freqs)
        assert np.linalg.norm(rb.coeffs - sig.coeffs[o]) < 16 * 2.0 ** -52 * math.sqrt(k) * 10
        assert sum(r["samples"] for r in rb.rounds) < sum(r["samples"] for r in rc.rounds)


def test_samples_equal_direct_real_point_evaluation():
    # f evaluated at the real point t = x u / p + s_n without any reduction (small numbers).
    sig = draw_signal(2, 16, 5, seed=3)
    p, u = 11, [1, 16]
    y = O.sample_sets(sig.freqs, sig.coeffs, p, u, 16)
    for n in range(3):
        for x in range(p):
            t = np.array([x * u[0] / p, x * u[1] / p]) + (np.eye(2)[n - 1] / 16 if n else 0)
            f = np.sum(sig.coeffs * np.exp(2j * np.pi * (sig.freqs @ t)))
            assert abs(y[n, x] - f) < 1e-11


# ---------------------------------------------------------------- DFT

def test_dft_equals_definition():
    for p in (2, 3, 5, 13, 61):
        rng = Stream(p)
        y = rng.uniform(3 * p).reshape(3, p) + 1j * rng.uniform(3 * p).reshape(3, p)
        F = np.array([[sum(y[r, x] * complex(math.cos(-2 * math.pi * h * x / p),
                                              math.sin(-2 * math.pi * h * x / p))
                            for x in range(p)) for h in range(p)] for r in range(3)])
        assert np.max(np.abs(O.dft(y) - F)) < 1e-11


def _check_single_mode_closed_form(sample_fn, dft_fn):
    # Eq. 3-5 and Eq. 41: one mode gives a single occupied bin h = (w . u) mod p holding
    # p a, and Y_n / Y_0 = exp(2 pi i w_n / N) there.
    d, N, p = 4, 1024, 83
    w = np.array([[700, 13, 1000, 512]])
    a = np.array([1.5 - 0.25j])
    u = [1, N, 0, 0]
    h = (700 + 13 * N) % p
    Y = dft_fn(sample_fn(w, a, p, u, N))
    assert abs(Y[0, h] - p * a[0]) < 1e-9
    Y0 = Y[0].copy()
    Y0[h] = 0
    assert np.max(np.abs(Y0)) < 1e-9
    for n in range(1, d + 1):
        assert abs(Y[n, h] / Y[0, h] - np.exp(2j * np.pi * w[0, n - 1] / N)) < 1e-12


def test_single_mode_closed_form():
    _check_single_mode_closed_form(O.sample_sets, O.dft)


def test_parseval_on_samples():
    sig = draw_signal(3, 256, 40, seed=5)
    y = O.sample_sets(sig.freqs, sig.coeffs, 211, [1, 256, 0], 256)
    Y = O.dft(y)
    lhs = np.sum(np.abs(y) ** 2, axis=1)
    rhs = np.sum(np.abs(Y) ** 2, axis=1) / 211
    assert np.allclose(lhs, rhs, rtol=1e-12)


# ---------------------------------------------------------------- registry in the bin domain

def _check_registry_bins(bins_fn):
    # (1) one mode: a delta at alpha = (w . u) mod p holding p a e^{2 pi i w_n / N} (closed form);
    # (2) modes sharing a bin add; (3) many modes: equal to the transform of their samples,
    # both pinned on their own above (brute-force rational points, the DFT definition).
    d, N, p = 4, 1024, 211
    u = [1, N, 0, 0]
    w = np.array([[700, 13, 1000, 512]])
    a = np.array([1.5 - 0.25j])
    h = (700 + 13 * N) % p
    G = bins_fn(w, a, p, u, N)
    assert G.shape == (d + 1, p)
    assert abs(G[0, h] - p * a[0]) < 1e-9
    for n in range(1, d + 1):
        assert abs(G[n, h] - p * a[0] * np.exp(2j * np.pi * w[0, n - 1] / N)) < 1e-9
    G[:, h] = 0
    assert np.max(np.abs(G)) == 0.0
    w2 = np.array([[3, 5, 0, 9], [3 + p, 5, 0, 9], [3, 5, 7, 9]])   # first two share a bin (and w_2..)
    a2 = np.array([1.0 + 1.0j, -0.5 + 2.0j, 0.25j])
    G2 = bins_fn(w2, a2, p, u, N)
    h2 = (3 + 5 * N) % p
    assert abs(G2[0, h2] - p * np.sum(a2)) < 1e-9
    assert abs(G2[1, h2] - p * (a2[0] * np.exp(2j * np.pi * 3 / N) + a2[1] * np.exp(2j * np.pi * (3 + p) / N)
                                + a2[2] * np.exp(2j * np.pi * 3 / N))) < 1e-9
    sig = draw_signal(d, N, 300, seed=77)
    G3 = bins_fn(sig.freqs, sig.coeffs, p, u, N)
    Y3 = O.dft(O.sample_sets(sig.freqs, sig.coeffs, p, u, N))
    assert np.max(np.abs(G3 - Y3)) < 1e-9 * p * np.sum(np.abs(sig.coeffs))


def test_registry_bins_equal_transform_of_registry_samples():
    _check_registry_bins(O.registry_bins)


def test_bin_domain_residual_recovers_the_same_result():
    # subtracting g after the transform (linearity) gives the same sets and, in FP64, the same
    # coefficients as subtracting it from the samples
    for d, N, k, blocks, seed in ((2, 1024, 16, (1, 1), 3), (5, 1024, 200, (3, 2), 4), (3, 256, 60, (3,), 5)):
        sig = draw_signal(d, N, k, seed=seed, r_lo=1.0, r_hi=10.0)
        th = O.Thresholds(tau=1e-7, rho=2.0 ** -40, delta=0.1)
        lit = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, th=th)
        bins = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, th=th, residual="bins")
        planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])]
        assert lit.converged and bins.converged
        assert np.array_equal(bins.freqs, planted) and np.array_equal(lit.freqs, planted)
        assert np.max(np.abs(bins.coeffs - lit.coeffs) / np.abs(lit.coeffs)) < 1e-12
        assert [r["p"] for r in bins.rounds] == [r["p"] for r in lit.rounds]
        assert all(rb["terms"] == k for rb in bins.rounds)


# ---------------------------------------------------------------- noise of the black box

def test_prime_floor_takes_the_ith_prime_above_the_floor():
    wl_sig = draw_signal(2, 1024, 16, seed=5, r_lo=1.0, r_hi=2.0)
    th = O.Thresholds(tau=1e-7, rho=2.0 ** -40, delta=0.1)
    res = O.multi_phaseshift(wl_sig.freqs, wl_sig.coeffs, 2, 1024, 16, (1, 1), th=th, p_min=1000)
    assert res.converged and np.array_equal(res.freqs, wl_sig.freqs[np.lexsort(wl_sig.freqs.T[::-1])])
    pr = _sieve(4000)
    for r in res.rounds:
        lo = max(5 * r["k_star"], 1000)
        assert r["p"] == int(pr[np.searchsorted(pr, lo) + r["round"] - 1])


STOP_RULE_W = np.array([[3, 5], [7, 5], [20, 30]], dtype=np.int64)
STOP_RULE_A = np.array([1.5 - 0.5j, -1.5 + 0.5j, 2.0 + 0.0j])


def _check_stop_rule(recover):
    # Modes 0 and 1 have opposite coefficients and differ only in coordinate 1, which lines along
    # e_2 do not see: on such a line they share a bin and cancel in set 0, while set 1 (shifted
    # along e_1) holds p a (e^{2 pi i 3/N} - e^{2 pi i 7/N}).  With every line along e_2 the pair
    # can never be separated: after mode 2 is found, set 0 is empty but the residual is not, so
    # the run must end unconverged instead of returning {mode 2} as the whole set.  Lines along
    # e_2 and e_1 in turn recover all three.
    N = 64
    conv, fw, fa = recover(STOP_RULE_W, STOP_RULE_A, N, dirs=[(0, 1)], max_rounds=8)
    assert not conv
    assert np.array_equal(fw, STOP_RULE_W[2:])
    conv, fw, fa = recover(STOP_RULE_W, STOP_RULE_A, N, dirs=None, max_rounds=0)
    order = np.lexsort(STOP_RULE_W.T[::-1])
    assert conv and np.array_equal(fw, STOP_RULE_W[order])
    return fa, STOP_RULE_A[order]


def test_stop_rule_reads_every_set():
    def recover(w, a, N, dirs, max_rounds):
        res = O.multi_phaseshift(w, a, 2, N, len(w), (1, 1), dirs=dirs, max_rounds=max_rounds or None,
                                 residual="bins")
        return res.converged, res.freqs, res.coeffs
    fa, ref = _check_stop_rule(recover)
    assert np.max(np.abs(fa - ref)) < 1e-12


SLIP_W = np.array([[100, 200, 300], [101, 200, 300], [5000, 6000, 7000]], dtype=np.int64)
SLIP_A = np.array([1.0 + 0.0j, -1.0 + 0.0j, 2.0 + 0.0j])
SLIP_N = 1 << 20
FLOAT_TH = dict(tau=1e-3, rho=2.0 ** -17, delta=0.25)


def _check_every_direction_stop(recover):
    # Modes 0 and 1 (+1 and -1) differ by one unit in coordinate 1 of N = 2^20: lines along e_2
    # and e_3 (rounds 1 and 2 with three blocks of one coordinate) put them in one bin, where
    # set 0 cancels and the shifted set of coordinate 1 holds only p |e^{2 pi i 100/N} -
    # e^{2 pi i 101/N}| = p 2 pi / N, below the float policies' empty-bin level (2^-17 of the
    # largest first-round bin, here mode 2's).  Round 2 finds no occupied bin of any set; only the
    # line along e_1 (round 3) separates the pair.  Every direction must come up empty before
    # the run stops.
    conv, fw, fa = recover(SLIP_W, SLIP_A, SLIP_N)
    order = np.lexsort(SLIP_W.T[::-1])
    assert conv and np.array_equal(fw, SLIP_W[order])
    return fa, SLIP_A[order]


def test_stop_rule_waits_for_every_line_direction():
    def recover(w, a, N):
        res = O.multi_phaseshift(w, a, 3, N, len(w), (1, 1, 1), th=O.Thresholds(**FLOAT_TH), residual="bins")
        assert [list(O.line_direction(3, N, (1, 1, 1), i)) for i in (1, 2, 3)] == [[0, 1, 0], [0, 0, 1], [1, 0, 0]]
        assert res.rounds[1]["accepted"] == 0 and res.rounds[2]["accepted"] == 2
        return res.converged, res.freqs, res.coeffs
    fa, ref = _check_every_direction_stop(recover)
    assert np.max(np.abs(fa - ref)) < 1e-12


def test_prime_rule_with_a_fractional_factor():
    # c = 5/2 and c = 3/8: round i takes the i-th prime at or above ceil(c k*), found by a sieve
    pr = _sieve(6000)
    for c, k, seed in ((2.5, 300, 7), (0.375, 40, 8)):
        sig = draw_signal(2, 1 << 12, k, seed=seed, r_lo=1.0, r_hi=10.0)
        res = O.multi_phaseshift(sig.freqs, sig.coeffs, 2, sig.N, k, (1, 1), c=c,
                                 th=O.Thresholds(tau=1e-7, rho=2.0 ** -40, delta=0.1), residual="bins")
        assert res.converged and np.array_equal(res.freqs, sig.freqs[np.lexsort(sig.freqs.T[::-1])])
        for r in res.rounds:
            lo = -(-int(c * 8) * r["k_star"] // 8)                 # ceil(c k*) in integers
            assert r["p"] == int(pr[np.searchsorted(pr, max(lo, 2)) + r["round"] - 1])


def test_philox_matches_the_published_known_answer_vectors():
    # the generator's authors' own test vectors: a swapped multiplier or key increment, a
    # permuted output word or a dropped round changes every one of them
    rows = _rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in v[:4]], v[4], v[5])
        assert [int(np.asarray(w).ravel()[0]) for w in out] == v[6:10]


def test_philox_is_a_bijection_with_full_avalanche():
    # for one key the 128-bit output of distinct counters never repeats; flipping one counter
    # bit flips about half of the 128 output bits (a dropped round, word or xor breaks one of these)
    n = 1 << 17
    c0 = np.arange(n, dtype=np.uint64)
    c1 = (np.arange(n, dtype=np.uint64) * np.uint64(7)) & np.uint64(0xFF)
    out = O.philox4x32_10(c0, c1, np.full(n, 5, np.uint64), np.zeros(n, np.uint64), 0x1234, 0xABCD)
    words = np.stack(out, axis=1).astype(np.uint64)
    assert np.unique(words, axis=0).shape[0] == n
    base = np.stack(O.philox4x32_10(c0[:4096], c1[:4096], 5, 0, 0x1234, 0xABCD), axis=1)
    for bit in (0, 13, 31):
        for word in range(4):
            cs = [c0[:4096], c1[:4096], np.full(4096, 5, np.uint64), np.zeros(4096, np.uint64)]
            cs[word] = cs[word] ^ np.uint64(1 << bit)
            flip = np.stack(O.philox4x32_10(*cs, 0x1234, 0xABCD), axis=1) ^ base
            bits = sum(bin(int(v)).count("1") for v in flip.reshape(-1)) / 4096.0
            assert abs(bits - 64.0) < 1.5
    assert np.array_equal(np.stack(O.philox4x32_10(c0[:64], c1[:64], 5, 0, 0x1234, 0xABCD)), base[:64].T)


def test_philox_words_are_uniform():
    n = 1 << 16
    out = O.philox4x32_10(np.arange(n, dtype=np.uint64), 3, 1, 0, 99, 7)
    for w in out:
        counts = np.bincount((w >> np.uint64(28)).astype(np.int64), minlength=16)
        chi2 = float(np.sum((counts - n / 16.0) ** 2 / (n / 16.0)))
        assert chi2 < 45.0          # 15 degrees of freedom: p < 2e-4 above this


def test_noise_is_complex_gaussian_with_the_stated_variance():
    sigma = 2e-3
    z = O.black_box_noise(0x9E3779B97F4A7C15, 3, 20011, 4, sigma)     # 100 055 samples
    assert z.shape == (5, 20011)
    re, im = z.real.reshape(-1), z.imag.reshape(-1)
    var = sigma ** 2 / 2
    sd_mean = math.sqrt(var / re.size)
    assert abs(re.mean()) < 5 * sd_mean and abs(im.mean()) < 5 * sd_mean
    assert abs(re.var() / var - 1) < 0.03 and abs(im.var() / var - 1) < 0.03
    assert abs(np.mean(re * im)) / var < 0.02                          # Re and Im independent
    assert abs(np.mean(re ** 4) / var ** 2 - 3.0) < 0.1                # Gaussian kurtosis
    # sets, points and rounds draw independent values
    assert abs(np.mean(z[0] * np.conj(z[1]))) / sigma ** 2 < 0.02
    assert abs(np.mean(z[:, 1:] * np.conj(z[:, :-1]))) / sigma ** 2 < 0.02
    z2 = O.black_box_noise(0x9E3779B97F4A7C15, 4, 20011, 4, sigma)
    assert abs(np.mean(z * np.conj(z2))) / sigma ** 2 < 0.02
    assert np.array_equal(z, O.black_box_noise(0x9E3779B97F4A7C15, 3, 20011, 4, sigma))


def test_noisy_recovery_errors_scale_like_sigma_over_root_p():
    # sigma = 1e-3 on modes of |a| in [1, 10]: the planted set is recovered and each coefficient
    # is off by about the noise of its bin, sigma / sqrt(p (d + 1)) for the mean over the sets
    d, N, k, sigma = 3, 256, 120, 1e-3
    sig = draw_signal(d, N, k, seed=41, r_lo=1.0, r_hi=10.0, noise_sigma=sigma)
    th = O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25, sigma=sigma)
    res = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, (2, 1), th=th, estimator="mean",
                             residual="bins",
                             noise=lambda i, p, dd: O.black_box_noise(sig.noise_seed, i, p, dd, sigma))
    order = np.lexsort(sig.freqs.T[::-1])
    assert res.converged and np.array_equal(res.freqs, sig.freqs[order])
    err = np.abs(res.coeffs - sig.coeffs[order])
    ps = [r["p"] for r in res.rounds]
    assert np.max(err) < 8 * sigma / math.sqrt(min(ps) * (d + 1))
    assert np.sqrt(np.mean(err ** 2)) > 0.2 * sigma / math.sqrt(max(ps) * (d + 1))   # the noise is there


# ---------------------------------------------------------------- bin test and decode

def _check_collision_rejected(classify_fn):
    # Two modes in one bin that differ in coordinate 2 only: Eq. 42 fails for n = 2 and the
    # bin is rejected.  A lone mode in another bin is read off exactly.
    d, N, p = 3, 64, 31
    u = [1, 0, 0]
    w = np.array([[5, 10, 7], [5, 40, 7], [20, 3, 60]])
    a = np.array([1.0 + 0.2j, 0.8 - 0.5j, -1.1 + 0.3j])
    Y = O.dft(O.sample_sets(w, a, p, u, N))
    acc = classify_fn(Y, p, u, N, 1e-6, O.Thresholds())
    assert [(h, wv) for h, wv, _ in acc] == [(20, (20, 3, 60))]
    assert abs(acc[0][2] - a[2]) < 1e-12


def test_collision_is_rejected_and_lone_mode_read_off():
    _check_collision_rejected(O.classify)


def test_mean_estimator_equals_eq41_on_single_mode_bins():
    # Every shifted set of a lone mode gives Y_n = p a e^{2 pi i w_n / N}: the mean estimator
    # returns a, and on whole recoveries both estimators agree to round-off.
    d, N, p = 3, 64, 31
    w = np.array([[20, 3, 60], [40, 33, 1]])
    a = np.array([-1.1 + 0.3j, 0.6 + 0.6j])
    Y = O.dft(O.sample_sets(w, a, p, [1, 0, 0], N))
    for est in ("set0", "mean"):
        acc = O.classify(Y, p, [1, 0, 0], N, 1e-6, O.Thresholds(), estimator=est)
        got = {wv: av for _, wv, av in acc}
        assert abs(got[(20, 3, 60)] - a[0]) < 1e-13 and abs(got[(40, 33, 1)] - a[1]) < 1e-13
    sig = draw_signal(3, 256, 60, seed=21)
    r0 = _recover(sig, (2, 1))
    r1 = _recover(sig, (2, 1), estimator="mean")
    assert np.array_equal(r0.freqs, r1.freqs) and np.max(np.abs(r0.coeffs - r1.coeffs)) < 1e-12


def test_arg_range_is_half_open():
    z = np.array([-1 + 0j, -1 - 1e-300j, 1j, -1j])
    a = O.arg(z)
    assert np.all(a >= -np.pi) and np.all(a < np.pi)
    assert a[0] == -np.pi


# ---------------------------------------------------------------- whole loop

def _recover(sig, blocks, **kw):
    return O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, blocks,
                              box_lo=sig.box_lo, **kw)


def _assert_exact(res, sig, tol):
    order = np.lexsort(sig.freqs.T[::-1])
    assert res.converged
    assert np.array_equal(res.freqs, sig.freqs[order].astype(np.int64))
    rel = np.abs(res.coeffs - sig.coeffs[order]) / np.abs(sig.coeffs[order])
    assert np.max(rel) < tol


def _check_full_grid(recover_fn):
    # The textbook d-dimensional FFT of f on its full grid is the ground truth.
    for d, N, k, seed in ((2, 32, 8, 1), (3, 16, 12, 2), (2, 64, 30, 3)):
        sig = draw_signal(d, N, k, seed=seed)
        F = O.full_grid_coefficients(sig.freqs, sig.coeffs, d, N)
        support = np.argwhere(np.abs(F) > 1e-9)
        res = recover_fn(sig)
        assert res.converged
        assert np.array_equal(res.freqs, support)          # argwhere is lexicographic
        assert np.max(np.abs(res.coeffs - F[tuple(support.T)])) < 1e-12


def test_recovery_equals_full_grid_fft():
    _check_full_grid(lambda s: _recover(s, (1,) * s.d))


def test_recovery_equals_full_grid_fft_signed_box():
    sig = draw_signal(2, 32, 10, seed=9, box_lo=-16)
    F = O.full_grid_coefficients(sig.freqs, sig.coeffs, 2, 32, box_lo=-16)
    support = np.argwhere(np.abs(F) > 1e-9) - 16
    res = _recover(sig, (1, 1))
    assert np.array_equal(res.freqs, support)


def test_workload_d2_recovers_planted_set():
    sig = draw_signal(2, 1024, 16, seed=1606074071, r_lo=1.0, r_hi=2.0)
    res = _recover(sig, (1, 1))
    _assert_exact(res, sig, 1e-12)
    assert res.rounds[0]["p"] == 83


def test_d5_full_unwrap_and_partial_unwrap():
    sig = draw_signal(5, 1024, 200, seed=77, r_lo=1, r_hi=10)
    _assert_exact(_recover(sig, (3, 2)), sig, 1e-12)
    _assert_exact(_recover(sig, (5,)), sig, 1e-12)


def test_d1_general_form_equals_algorithm_1():
    sig = draw_signal(1, 4096, 40, seed=4)
    w1, a1 = O.phaseshift_1d(sig.freqs[:, 0], sig.coeffs, 4096, 40)
    res = _recover(sig, (1,))
    assert np.array_equal(res.freqs[:, 0], w1)
    # Alg. 1 as printed evaluates f at the unreduced real point t, whose phase 2 pi w t
    # reaches 2 pi N: its double rounding is about N * 2 pi * 2^-53 ~ 3e-12 per term.
    assert np.max(np.abs(res.coeffs - a1)) < 1e-10
    _assert_exact(res, sig, 1e-12)


def test_4d_two_by_two_example():
    sig = draw_signal(4, 32, 60, seed=8)
    _assert_exact(_recover(sig, (2, 2)), sig, 1e-12)


def test_fig2_collision_story():
    rows = _rows("fig2_collisions.txt")
    w = np.array([[int(r[1]), int(r[2])] for r in rows])
    a = np.array([float(r[3]) + 1j * float(r[4]) for r in rows])
    # round i uses dirs[i mod 2]: round 1 projects on the horizontal axis, round 2 on the vertical.
    res = O.multi_phaseshift(w, a, 2, 16, 3, dirs=[[0, 1], [1, 0]], primes=[17, 17, 17, 17])
    assert res.rounds[0]["accepted"] == 1 and res.rounds[0]["registry"] == 1
    assert res.rounds[1]["accepted"] == 2 and res.rounds[1]["registry"] == 3
    assert res.converged and res.n_found == 3


def test_paper_workload_shape_error_below_claim():
    # Sec. 5 / Sec. 5.1: d = 100, d1 = 5, d2 = 20, N = 20, |a_j| = 1, box [-N/2, N/2)^d;
    # frequencies exact and the l2 coefficient error at double round-off (the paper reports
    # an average below 2^-52; a few ulps per coefficient are allowed here).
    for k, seed in ((1, 1), (4, 2), (16, 3)):
        sig = draw_signal(100, 20, k, seed=seed, box_lo=-10, unit_modulus=True)
        res = _recover(sig, (5,) * 20)
        order = np.lexsort(sig.freqs.T[::-1])
        assert np.array_equal(res.freqs, sig.freqs[order].astype(np.int64))
        err = np.linalg.norm(res.coeffs - sig.coeffs[order])
        assert err < 16 * 2.0 ** -52 * math.sqrt(k)


def test_sample_count_grows_like_d_times_k():
    # Theorem 3: E[S(k)] = Theta(d k).  Samples / (d k) stays in a narrow band.
    ratios = []
    for d, k in ((2, 8), (2, 64), (4, 64), (4, 256)):
        sig = draw_signal(d, 1 << 12, k, seed=d * 1000 + k)
        res = _recover(sig, (1,) * d if d == 2 else (2, 2))
        ratios.append(res.samples / ((d + 1) * k))
    assert max(ratios) / min(ratios) < 4.0 and min(ratios) > 5.0


# ---------------------------------------------------------------- the pins catch slips

def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle and check that some pin fails for each."""
    real_sample = O.sample_sets
    real_classify = O.classify

    def wrong_sign(freqs, coeffs, p, u, N):      # e^{-2 pi i ...} in the black box
        return np.conj(real_sample(freqs, np.conj(coeffs), p, u, N))

    def dropped_shift(freqs, coeffs, p, u, N):   # the shift term w_n / N left out
        y = real_sample(freqs, coeffs, p, u, N)
        y[1:] = y[0]
        return y

    def transposed_u(freqs, coeffs, p, u, N):    # direction applied to the wrong coordinates
        return real_sample(freqs, coeffs, p, list(u)[::-1], N)

    def off_by_one_shift(freqs, coeffs, p, u, N):   # shift along e_{n+1} instead of e_n
        y = real_sample(freqs, coeffs, p, u, N)
        return np.concatenate([y[:1], np.roll(y[1:], 1, axis=0)])

    for bad in (wrong_sign, dropped_shift, transposed_u, off_by_one_shift):
        with pytest.raises(AssertionError):
            _check_samples_against_rationals(bad)
        with pytest.raises(AssertionError):
            _check_single_mode_closed_form(bad, O.dft)

    def ratio_inverted(Y, p, u, N, eta, th, box_lo=0):   # Arg of Y_0 / Y_n (sign slip)
        return real_classify(np.concatenate([Y[:1], np.conj(Y[1:]) * (Y[:1] / np.conj(Y[:1]))]),
                             p, u, N, eta, th, box_lo)

    def no_ratio_test(Y, p, u, N, eta, th, box_lo=0):
        return real_classify(Y, p, u, N, eta, O.Thresholds(tau=1e9, delta=0.5), box_lo)

    for bad in (ratio_inverted, no_ratio_test):
        with pytest.raises(AssertionError):
            _check_collision_rejected(bad)

    def coeff_conj(sig):                           # a = conj(Y_0)/p
        res = _recover(sig, (1,) * sig.d)
        res.coeffs = np.conj(res.coeffs)
        return res

    with pytest.raises(AssertionError):
        _check_full_grid(coeff_conj)

    real_bins = O.registry_bins

    def bins_no_p(freqs, coeffs, p, u, N):          # the factor p of the DFT dropped
        return real_bins(freqs, coeffs, p, u, N) / p

    def bins_conj_phase(freqs, coeffs, p, u, N):    # e^{-2 pi i w_n / N} on the shifted sets
        return np.conj(real_bins(freqs, np.conj(coeffs), p, u, N))

    def bins_wrong_bin(freqs, coeffs, p, u, N):     # off-by-one bin index
        return np.roll(real_bins(freqs, coeffs, p, u, N), 1, axis=1)

    for bad in (bins_no_p, bins_conj_phase, bins_wrong_bin):
        with pytest.raises(AssertionError):
            _check_registry_bins(bad)

    real_phases = O.shift_phases

    def eps_not_halved(freqs, N, shift="coord", blocks=None, tilt=None):   # eps = 1 / N^{d1}: read-out wraps
        num, q = real_phases(freqs, N, shift, blocks, tilt)
        if shift == "block":
            q = q // 2
            num = np.mod(num, q[None, :])
        return num, q

    monkeypatch.setattr(O, "shift_phases", eps_not_halved)
    with pytest.raises(AssertionError):
        test_block_readout_decodes_every_vector_of_a_box()
    with pytest.raises(AssertionError):
        _check_block_samples_against_rationals(
            lambda f, a, p, u, N: O.sample_sets(f, a, p, u, N, shift="block", blocks=(2, 3)))
    monkeypatch.setattr(O, "shift_phases", real_phases)

    real_axes = O.tilt_axes

    def axes_unsigned(tilt):                       # rotated axis 1 taken as (base, height)
        return np.abs(real_axes(tilt))

    def axes_swapped(tilt):                        # the two rotated axes exchanged
        return real_axes(tilt)[::-1].copy()

    for bad in (axes_unsigned, axes_swapped):
        monkeypatch.setattr(O, "tilt_axes", bad)
        with pytest.raises(AssertionError):
            _check_tilt_samples_against_rationals(
                lambda f, a, p, u, N: O.sample_sets(f, a, p, u, N, shift="tilt", tilt=TILT_16))
        monkeypatch.setattr(O, "tilt_axes", real_axes)

    real_window = O.tilt_window

    def window_unsigned(N, box_lo, tilt):          # the first rotated coordinate's window from 0
        Q, lo = real_window(N, box_lo, tilt)
        return Q, (0, lo[1])

    monkeypatch.setattr(O, "tilt_window", window_unsigned)
    with pytest.raises(AssertionError):
        test_tilt_readout_decodes_every_pair_of_a_box_and_rejects_the_rest()
    monkeypatch.setattr(O, "tilt_window", real_window)

    real_core = O.projection_core

    def core_one_pass(freqs, N, blocks, box_lo=0):   # each block peeled once, no repeat
        wt = O.unwrapped_coordinates(freqs, N, blocks, box_lo)
        alive = set(range(wt.shape[0]))
        for q in range(wt.shape[1]):
            count = {}
            for j in alive:
                count[wt[j, q]] = count.get(wt[j, q], 0) + 1
            alive -= {j for j in alive if count[wt[j, q]] == 1}
        return np.array(sorted(alive), dtype=np.int64)

    def core_counts_once(freqs, N, blocks, box_lo=0):   # shared values counted over all modes only
        wt = O.unwrapped_coordinates(freqs, N, blocks, box_lo)
        K, B = wt.shape
        keep = [j for j in range(K) if all(sum(wt[i, q] == wt[j, q] for i in range(K)) > 1 for q in range(B))]
        return np.array(keep, dtype=np.int64)

    for bad in (core_one_pass, core_counts_once):
        monkeypatch.setattr(O, "projection_core", bad)
        with pytest.raises(AssertionError):
            test_projection_core_in_two_dimensions_is_the_two_core_of_the_row_column_graph()
        with pytest.raises(AssertionError):
            test_parallel_projections_fail_exactly_on_the_projection_core()
        monkeypatch.setattr(O, "projection_core", real_core)

    real_decode_tilt = O._decode_tilt

    def tilt_turned_the_wrong_way(ratio, N, tilt, box_lo, delta):   # [cos -sin; sin cos] back
        return real_decode_tilt(ratio, N, (tilt[0], -tilt[1], tilt[2]), box_lo, delta)

    monkeypatch.setattr(O, "_decode_tilt", tilt_turned_the_wrong_way)
    with pytest.raises(AssertionError):
        test_tilt_readout_decodes_every_pair_of_a_box_and_rejects_the_rest()
    monkeypatch.setattr(O, "_decode_tilt", real_decode_tilt)

    real_philox = O.philox4x32_10

    def philox_2_rounds(c0, c1, c2, c3, k0, k1):       # two rounds, no key schedule: weak mixing
        c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & np.uint64(0xFFFFFFFF) for v in (c0, c1, c2, c3))
        out = (c0, c1, c2, c3)
        k0, k1 = np.uint64(k0), np.uint64(k1)
        for rnd in range(2):
            p0, p1 = out[0] * np.uint64(0xD2511F53), out[2] * np.uint64(0xCD9E8D57)
            out = ((p1 >> np.uint64(32)) ^ out[1] ^ k0, p1 & np.uint64(0xFFFFFFFF),
                   (p0 >> np.uint64(32)) ^ out[3] ^ k1, p0 & np.uint64(0xFFFFFFFF))
        return out

    monkeypatch.setattr(O, "philox4x32_10", philox_2_rounds)
    with pytest.raises(AssertionError):
        test_philox_is_a_bijection_with_full_avalanche()
    monkeypatch.setattr(O, "philox4x32_10", real_philox)

    def philox_variant(m0, m1, w0, w1, perm):
        # Philox4x32-10 with its constants or output order changed: each of these still mixes
        # fully, so only the published vectors tell it from the generator
        def gen(c0, c1, c2, c3, k0, k1):
            m32 = np.uint64(0xFFFFFFFF)
            c = [np.asarray(v, dtype=np.uint64) & m32 for v in (c0, c1, c2, c3)]
            ka, kb = np.uint64(int(k0) & 0xFFFFFFFF), np.uint64(int(k1) & 0xFFFFFFFF)
            for rnd in range(10):
                if rnd:
                    ka, kb = (ka + np.uint64(w0)) & m32, (kb + np.uint64(w1)) & m32
                p0, p1 = c[0] * np.uint64(m0), c[2] * np.uint64(m1)
                c = [(p1 >> np.uint64(32)) ^ c[1] ^ ka, p1 & m32, (p0 >> np.uint64(32)) ^ c[3] ^ kb, p0 & m32]
            return tuple(c[i] for i in perm)
        return gen

    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    monkeypatch.setattr(O, "philox4x32_10", philox_variant(M0, M1, W0, W1, (0, 1, 2, 3)))
    test_philox_matches_the_published_known_answer_vectors()       # the restatement itself passes
    for bad in (philox_variant(M1, M0, W0, W1, (0, 1, 2, 3)),      # multipliers swapped
                philox_variant(M0, M1, W1, W0, (0, 1, 2, 3)),      # key increments swapped
                philox_variant(M0, M1, W0, W1, (1, 0, 3, 2))):     # output words permuted
        monkeypatch.setattr(O, "philox4x32_10", bad)
        test_philox_is_a_bijection_with_full_avalanche()           # the statistical pins miss it
        with pytest.raises(AssertionError):
            test_philox_matches_the_published_known_answer_vectors()
    monkeypatch.setattr(O, "philox4x32_10", real_philox)

    real_noise = O.black_box_noise
    monkeypatch.setattr(O, "black_box_noise", lambda seed, i, p, d, sigma: real_noise(seed, i, p, d, sigma * 2 ** 0.5))
    with pytest.raises(AssertionError):                 # sigma per component instead of sigma / sqrt 2
        test_noise_is_complex_gaussian_with_the_stated_variance()
    monkeypatch.setattr(O, "black_box_noise", real_noise)
