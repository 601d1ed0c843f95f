"""Host-side helpers of the experiment modules (CPU only): the bound of Sec. 4.2 and the pair
event as the worst-case experiment computes them, against the oracle and brute force, and the
rectangle-corner generator of the tilted-lines experiment."""
import itertools

import numpy as np

import oracle.sfft_oracle as O
from paper_1606_07407_gb300.inputs import draw_rectangle_signal, draw_signal
from paper_1606_07407_gb300.worst_case_experiment import CASES, pair_on_common_line, paper_bound, wilson


def test_bound_matches_the_oracle_on_every_case():
    for d, N, blocks, ks in CASES:
        for k in ks:
            assert abs(paper_bound(N, blocks, k) - O.worst_case_bound(N, blocks, k)) < 1e-9


def test_pair_event_matches_brute_force():
    # two vectors share an axis-parallel line of the unwrapped coordinates when they agree on
    # every block's unwrapped value but one
    for d, N, blocks, k, seeds in ((2, 8, (1, 1), 5, 30), (4, 4, (2, 2), 6, 30), (3, 4, (1, 1, 1), 5, 30)):
        for seed in range(seeds):
            w = draw_signal(d, N, k, seed=900 + seed).freqs
            wt = O.unwrapped_coordinates(w, N, blocks)
            want = any(sum(wt[i, q] != wt[j, q] for q in range(len(blocks))) == 1
                       for i, j in itertools.combinations(range(k), 2))
            assert pair_on_common_line(w, N, blocks) == want


def test_wilson_interval_brackets_the_share():
    for x, n in ((0, 100), (3, 100), (50, 100), (100, 100)):
        lo, hi = wilson(x, n)
        assert 0.0 <= lo <= x / n <= hi <= 1.0


def test_rectangle_signal_puts_every_corner_in_the_projection_core():
    for seed in range(10):
        sig = draw_rectangle_signal(64, 60, 10, seed=seed)
        assert len({tuple(w) for w in sig.freqs.tolist()}) == 60
        core = set(O.projection_core(sig.freqs, 64, (1, 1)).tolist())
        assert set(range(40)) <= core


def test_tilt_experiment_triples_meet_theorem_1():
    # each case's triple is primitive Pythagorean with base > 2N, so the rotated coordinates of
    # the box are distinct (Theorem 1), and its read-out fits the case's precision policy
    from paper_1606_07407_gb300.tilt_experiment import CASES as TILT_CASES
    for N, prec, tilt, k, n_rect, div in TILT_CASES:
        O.check_tilt(tilt)
        base, height, _ = tilt
        assert base > 2 * N and 4 * n_rect <= k
        Q, _ = O.tilt_window(N, 0, tilt)
        assert prec == "fp64" or Q <= 2 ** 21
