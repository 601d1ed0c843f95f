"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Step by step: samples of kernel (a), DFTs of kernel (b), bin read-out of kernel
(c); then whole recoveries, where the recovered frequency set must equal the
oracle's and the planted set exactly and the coefficients agree within 1e-5
relative (FP32 bulk) or 1e-12 (FP64).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.sfft_oracle as O
from paper_1606_07407_gb300.inputs import WORKLOADS, Stream, draw_rectangle_signal, draw_signal

pytestmark = pytest.mark.gpu

FP32_COEFF_TOL = 1e-5
FP64_COEFF_TOL = 1e-12
# DF64 (double-float sampling, about 48 significant bits): a sample's error is at most about
# 2^-46 of sum |a| per operation on its path (8 per term, then the additions of a 32-mode chunk
# and of the K / 32 chunk sums); a coefficient from p samples then errs by about that over
# sqrt(p) |a|, so 1e-10 relative leaves a wide margin at the test sizes
DF64_COEFF_TOL = 1e-10


def _df64_sample_tol(K, coeffs):
    return (8 + 32 + math.ceil(K / 32)) * 2.0 ** -46 * np.sum(np.abs(coeffs))


def _double(prec):
    return prec in ("fp64", "df64")


def _sample_tol(prec, K, coeffs):
    if prec == "df64":
        return _df64_sample_tol(K, coeffs)
    return (2.0 ** -20 if prec == "fp32" else 2.0 ** -48) * np.sum(np.abs(coeffs))
# the FP64 policy ends a recovery after one empty round (its read-outs do not slip); the float
# policies after one per line direction (the oracle's default)
FP64_EMPTY_ROUNDS = 1


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1606_07407_gb300 import build as B
    B.build()
    from paper_1606_07407_gb300 import sfft as S
    S.load()
    return S


def _np(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ kernel (a)

@pytest.mark.parametrize("prec", ["fp32", "fp64", "df64"])
@pytest.mark.parametrize("d,N,K,p,blocks", [
    (2, 1024, 16, 83, (1, 1)),        # one tile, one mode chunk
    (3, 4096, 100, 1031, (2, 1)),      # 3 tiles (ragged), 4 mode chunks (ragged)
    (5, 1024, 1000, 5003, (3, 2)),     # first round of the d=5 workload
    (12, 256, 70, 211, (3,) * 4),      # 13 sets: two set groups
])
def test_samples_match_oracle(sfft, prec, d, N, K, p, blocks):
    sig = draw_signal(d, N, K, seed=1000 + K, r_lo=1.0, r_hi=10.0)
    plan = sfft.Plan(d, N, max(K, 16), blocks=blocks, precision=prec)
    for m in range(len(blocks)):
        u = [int(v) for v in O.unwrap_vector(d, N, blocks, m)]
        y = _np(plan.sample(p, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs)))
        ref = O.sample_sets(sig.freqs, sig.coeffs, p, u, N)
        assert np.max(np.abs(y - ref)) < _sample_tol(prec, K, sig.coeffs)


def test_samples_registry_sign_and_empty(sfft):
    # K = 0 gives exact zeros; negated coefficients give negated samples (f - g).
    plan = sfft.Plan(2, 64, 8, blocks=(1, 1))
    y0 = _np(plan.sample(13, [1, 0], torch.zeros((0, 2), dtype=torch.int32), torch.zeros(0, dtype=torch.complex128)))
    assert np.all(y0 == 0)
    w = torch.tensor([[3, 5], [7, 60]], dtype=torch.int32)
    a = torch.tensor([1 + 1j, -0.5 + 2j], dtype=torch.complex128)
    yp, ym = _np(plan.sample(13, [1, 0], w, a)), _np(plan.sample(13, [1, 0], w, -a))
    assert np.max(np.abs(yp + ym)) == 0.0


def test_samples_sampled_at_large_size(sfft):
    # d = 10, N = 2^16, K = 10000 modes, p = 50021: compare 64 sampled columns.
    sig = draw_signal(10, 1 << 16, 10000, seed=3, r_lo=1.0, r_hi=10.0)
    blocks = (2,) * 5
    plan = sfft.Plan(10, 1 << 16, 10000, blocks=blocks)
    u = [int(v) for v in O.unwrap_vector(10, 1 << 16, blocks, 1)]
    y = _np(plan.sample(50021, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs)))
    xs = np.array(sorted(set(Stream(5).integers(64, 0, 50021).tolist()) | {0, 50020}))
    ref = O.sample_sets(sig.freqs, sig.coeffs, 50021, u, 1 << 16, x_values=xs)
    assert np.max(np.abs(y[:, xs] - ref)) < 2.0 ** -20 * np.sum(np.abs(sig.coeffs))


# ------------------------------------------------------------------ kernel (b)

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("p", [2, 5, 83, 911, 2039, 4099, 5003, 8191, 8209, 50021])
def test_dft_matches_definition(sfft, prec, p):
    # one-block Bluestein up to L = 16384 in float (p = 8191) and L = 10240 = 5 * 2^11 in double
    # (p = 4099, beyond the one-block limit of 8192 there: four-step); p = 8209 and 50021 take the
    # four-step passes.
    rows = 3
    plan = sfft.Plan(2, 1 << 16, 12000, blocks=(1, 1), precision=prec)
    st = Stream(p)
    y = (st.uniform(rows * p) - 0.5 + 1j * (st.uniform(rows * p) - 0.5)).reshape(rows, p)
    Yg = _np(plan.dft(p, torch.tensor(y)))
    ycast = y.astype(np.complex64).astype(np.complex128) if prec == "fp32" else y
    ref = O.dft(ycast)
    L = 1 << math.ceil(math.log2(2 * p - 1))
    eps = 2.0 ** -24 if prec == "fp32" else 2.0 ** -53
    for r in range(rows):
        tol = 16 * eps * math.log2(L) * np.linalg.norm(ycast[r])
        assert np.max(np.abs(Yg[r] - ref[r])) < tol


def _primes_upto(n):
    s = np.ones(n + 1, dtype=bool)
    s[:2] = False
    for q in range(2, int(n ** 0.5) + 1):
        if s[q]:
            s[q * q::q] = False
    return np.nonzero(s)[0]


def _length_classes(lmax):
    # the convolution lengths m 2^a (m = 1, 3, 5; 32 <= L <= lmax) and, for each, the largest
    # prime p whose 2p - 1 falls between it and the next smaller length: that p uses it
    Ls = sorted({m << a for m in (1, 3, 5) for a in range(0, 15) if 32 <= (m << a) <= lmax})
    pr = _primes_upto(lmax)
    out, prev = [], 0
    for L in Ls:
        cand = [int(q) for q in pr if prev < 2 * q - 1 <= L]
        if cand:
            out.append((L, cand[-1]))
        prev = L
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_dft_every_bluestein_length(sfft, prec):
    # every pass shape of the one-block FFT: powers of two, 3 2^a and 5 2^a, with the odd factor
    # in a combined radix-(m 2^b) pass or a separate radix-m pass, in both block classes
    lmax = 16384 if prec == "fp32" else 8192
    plan = sfft.Plan(2, 1 << 16, 12000, blocks=(1, 1), precision=prec)
    eps = 2.0 ** -24 if prec == "fp32" else 2.0 ** -53
    classes = _length_classes(lmax)
    assert len(classes) >= 25
    for L, p in classes:
        st = Stream(L)
        y = (st.uniform(2 * p) - 0.5 + 1j * (st.uniform(2 * p) - 0.5)).reshape(2, p)
        Yg = _np(plan.dft(p, torch.tensor(y)))
        ycast = y.astype(np.complex64).astype(np.complex128) if prec == "fp32" else y
        ref = O.dft(ycast)
        for r in range(2):
            tol = 16 * eps * math.log2(L) * np.linalg.norm(ycast[r])
            assert np.max(np.abs(Yg[r] - ref[r])) < tol, (L, p)


def test_dft_single_mode_closed_form(sfft):
    # Eq. 3-5: samples of one mode transform to p a at its bin and ~0 elsewhere.
    p, N = 5003, 1024
    plan = sfft.Plan(5, N, 1000, blocks=(3, 2))
    w = torch.tensor([[700, 13, 1000, 512, 9]], dtype=torch.int32)
    a = torch.tensor([1.5 - 0.25j], dtype=torch.complex128)
    u = [1, N, N * N, 0, 0]
    Y = _np(plan.dft(p, plan.sample(p, u, w, a)))
    h = (700 + 13 * N + 1000 * N * N) % p
    assert abs(Y[0, h] - p * a[0].item()) < 1e-5 * p
    mask = np.ones(p, bool)
    mask[h] = False
    assert np.max(np.abs(Y[:, mask])) < 1e-5 * p
    for n in range(1, 6):
        assert abs(Y[n, h] / Y[0, h] - np.exp(2j * np.pi * int(w[0, n - 1]) / N)) < 1e-6


def test_dft_large_prime_sampled(sfft):
    # the largest lengths a d=20, N=2^20, k=10^5 plan reaches (L = 2^20): sampled bins
    p = 500009
    plan = sfft.Plan(1, 1 << 20, 100000, blocks=(1,))
    st = Stream(9)
    y = (st.uniform(p) - 0.5 + 1j * (st.uniform(p) - 0.5)).reshape(1, p)
    Yg = _np(plan.dft(p, torch.tensor(y)))
    yc = y.astype(np.complex64).astype(np.complex128)[0]
    hs = np.array([0, 1, 2, 77777, p // 2, p - 1])
    x = np.arange(p)
    for h in hs:
        ref = np.sum(yc * np.exp(-2j * np.pi * ((h * x) % p) / p))
        assert abs(Yg[0, h] - ref) < 16 * 2.0 ** -24 * 20 * np.linalg.norm(yc)


# ------------------------------------------------------------------ kernel (c)

def _designed_transforms(d, N, p, u, w, a):
    return O.dft(O.sample_sets(np.array(w), np.array(a), p, u, N))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_classify_matches_oracle(sfft, prec):
    d, N, p = 3, 64, 31
    u = [1, 0, 0]
    # bin 5: two modes differing in coordinate 2 (rejected); bins 20, 9: lone modes;
    # bin 12: two modes differing in coordinate 1 by p (rejected)
    w = [[5, 10, 7], [5, 40, 7], [20, 3, 60], [40, 33, 1], [12, 0, 0], [43, 0, 0]]
    a = [1.0 + 0.2j, 0.8 - 0.5j, -1.1 + 0.3j, 0.6 + 0.6j, 1.0, 0.7j]
    Y = _designed_transforms(d, N, p, u, w, a)
    plan = sfft.Plan(d, N, 16, blocks=(1, 1, 1), precision="fp32_fp64ratio" if prec == "fp32" else prec)
    Yc = Y.astype(np.complex64 if prec == "fp32" else np.complex128)
    h, gw, ga = plan.classify(p, u, torch.tensor(Yc), 1e-3)
    th = O.Thresholds(tau=plan_tau(prec), delta=plan_delta(prec))
    ref = O.classify(Yc.astype(np.complex128), p, u, N, 1e-3, th, estimator="mean")
    got = sorted(zip(_np(h).tolist(), map(tuple, _np(gw).tolist()), _np(ga).tolist()))
    assert [(x[0], x[1]) for x in got] == [(r[0], r[1]) for r in ref] == [(9, (40, 33, 1)), (20, (20, 3, 60))]
    for g, r in zip(got, ref):
        assert abs(g[2] - r[2]) <= 1e-12 * abs(r[2])


@pytest.mark.parametrize("N", [1 << 20, 1 << 23, 999_983])
def test_classify_double_readout_at_large_N(sfft, N):
    # The float policies' double read-out (phase reduced against a table of 1024th turns, then a
    # short series) and table-based coefficient roots, at N where float's phase resolution no
    # longer reads a coordinate: 300 lone modes in distinct bins, float transforms of them, the
    # same accepted (bin, vector) set as the FP64 oracle on the same values and coefficients
    # within 1e-12 of its
    d, p, k = 3, 1031, 300
    u = [1, 0, 0]
    st = Stream(N % 1000 + 5)
    bins = np.unique(st.integers(4 * k, 0, p))[:k]
    rows = []
    for b in bins.tolist():
        w0 = b + p * int(st.integers(1, 0, (N - b) // p)[0])
        rows.append([w0, int(st.integers(1, 0, N)[0]), int(st.integers(1, 0, N)[0])])
    w = np.array(rows, dtype=np.int64)
    a = (1.0 + 9.0 * st.uniform(len(rows))) * np.exp(2j * np.pi * st.uniform(len(rows)))
    Yc = _designed_transforms(d, N, p, u, w, a).astype(np.complex64)
    plan = sfft.Plan(d, N, k, blocks=(1, 1, 1), precision="fp32_fp64ratio")
    eta = 2.0 ** -17 * np.max(np.abs(Yc[0]))
    h, gw, ga = plan.classify(p, u, torch.tensor(Yc), eta)
    ref = O.classify(Yc.astype(np.complex128), p, u, N, eta, O.Thresholds(tau=1e-3, delta=0.25), estimator="mean")
    got = sorted(zip(_np(h).tolist(), map(tuple, _np(gw).tolist()), _np(ga).tolist()))
    assert [(x[0], x[1]) for x in got] == [(r[0], r[1]) for r in ref]
    assert len(got) > k // 2
    for g, r in zip(got, ref):
        assert abs(g[2] - r[2]) <= 1e-12 * abs(r[2])


def plan_tau(prec):
    return 1e-7 if prec == "fp64" else 1e-3


def plan_delta(prec):
    return 0.1 if prec == "fp64" else 0.25


def test_classify_random_round_matches_oracle(sfft):
    # a first round of the d=5 workload: the accepted (bin, vector) sets are identical
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal()
    p = 5003
    u = [int(v) for v in O.unwrap_vector(5, 1024, wl.blocks, 1)]
    # read-out decisions in double on both sides (the oracle's precision)
    plan = sfft.Plan(5, 1024, 1000, blocks=wl.blocks, precision="fp32_fp64ratio")
    Y = _np(plan.dft(p, plan.sample(p, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs))))
    eta = 2.0 ** -17 * np.max(np.abs(Y[0]))
    h, gw, ga = plan.classify(p, u, torch.tensor(Y), eta)
    ref = O.classify(Y.astype(np.complex128), p, u, 1024, eta, O.Thresholds(tau=1e-3, delta=0.25))
    got = sorted(zip(_np(h).tolist(), map(tuple, _np(gw).tolist())))
    assert got == [(r[0], r[1]) for r in ref]
    assert len(got) > 700
    planted = {tuple(r) for r in sig.freqs.tolist()}
    assert all(g[1] in planted for g in got)


# ------------------------------------------------------------------ whole recovery

def _run_both(sfft, sig, blocks=None, prec="fp32", dirs=None, primes=None, box_lo=0, residual="bins", fuse=True,
              graph=False):
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=blocks, dirs=dirs, primes=primes, precision=prec, box_lo=box_lo,
                     residual=residual, fuse=fuse, graph=graph)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    th = O.Thresholds() if _double(prec) else O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, blocks, th=th, dirs=dirs,
                             empty_rounds=FP64_EMPTY_ROUNDS if _double(prec) else None,
                             primes=primes, box_lo=box_lo, estimator="mean", residual=residual)
    return gf, ga, status, stats, ref


def _assert_parity(sig, gf, ga, status, stats, ref, tol):
    planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
    assert status == 0 and stats["converged"] and ref.converged
    assert np.array_equal(gf, ref.freqs)
    assert np.array_equal(gf, planted)
    rel = np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)
    assert np.max(rel) < tol
    assert stats["p"] == [r["p"] for r in ref.rounds]


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_recovery_d2_workload(sfft, seed):
    wl = WORKLOADS["d2_N1024_k16"]
    sig = wl.signal(seed_offset=seed * 101)
    _assert_parity(sig, *_run_both(sfft, sig, wl.blocks), FP32_COEFF_TOL)


@pytest.mark.parametrize("residual", ["bins", "samples"])
def test_recovery_d5_workload_full_size(sfft, residual):
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal()
    _assert_parity(sig, *_run_both(sfft, sig, wl.blocks, residual=residual), FP32_COEFF_TOL)


@pytest.mark.parametrize("residual", ["bins", "samples"])
def test_fused_short_rounds_match_oracle_and_cut_launches(sfft, residual):
    # rounds on short lines run one block per signal in the fused kernel (default) or through
    # the batched kernels (fuse=False): both reach the oracle's result, the fused one in a third
    # fewer launches or less (graph mode counts the launches its loops ran; the rounds on long
    # lines and the launches around the loop are the same for both)
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=5)
    launches = {}
    for fuse in (True, False):
        out = _run_both(sfft, sig, wl.blocks, residual=residual, fuse=fuse, graph=True)
        _assert_parity(sig, *out, FP32_COEFF_TOL)
        launches[fuse] = sum(out[3]["launches"].values())
    assert 3 * launches[True] <= 2 * launches[False]


def test_fused_rounds_with_a_registry_too_large_for_shared_memory(sfft):
    # d = 2 (3 sets), k = 20000: the fused rounds' registry (about k entries) exceeds the shared
    # list of entry bins (15360 for 3 sets), so they take the whole registry off every set with
    # atomics instead of set 0 first; both paths recover the planted set
    sig = draw_signal(2, 4096, 20000, seed=20000, r_lo=1.0, r_hi=10.0)
    order = np.lexsort(sig.freqs.T[::-1])
    planted, a_true = sig.freqs[order].astype(np.int64), sig.coeffs[order]
    got = {}
    for fuse in (True, False):
        plan = sfft.Plan(2, 4096, 20000, blocks=(2,), fuse=fuse)   # full unwrap: N^2 >= p
        f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
        gf, ga = sfft.sort_result(_np(f), _np(a))
        assert status == 0 and np.array_equal(gf, planted)
        assert np.max(np.abs(ga - a_true) / np.abs(a_true)) < 1e-4
        got[fuse] = stats
    assert got[True]["terms_fused"] > 0 and got[False]["terms_fused"] == 0


def test_residual_forms_count_their_sample_terms(sfft):
    # bins: every round sums the black box's k modes; samples: k plus every registry entry
    # made so far (pruned ones included), so from round 2 on more than k + the live count
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=3)
    out = {}
    for residual in ("bins", "samples"):
        plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, residual=residual)
        f, a, status, st = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
        assert status == 0
        R = st["rounds"]
        assert st["samples"] == sum((wl.d + 1) * p for p in st["p"][:R])
        assert st["terms"] == sum((wl.d + 1) * p * K for p, K in zip(st["p"][:R], st["K"][:R]))
        out[residual] = st
    b, s_ = out["bins"], out["samples"]
    assert b["p"] == s_["p"] and b["accepted"] == s_["accepted"]
    assert all(K == wl.k for K in b["K"][:b["rounds"]])
    assert s_["K"][0] == wl.k
    assert all(K >= wl.k + live for K, live in zip(s_["K"][1:s_["rounds"]], s_["registry"]))
    assert b["terms"] < s_["terms"]


@pytest.mark.parametrize("case", ["d1", "d4_2x2", "d3_full_unwrap", "d6_tilted", "signed_box", "d12"])
def test_recovery_shapes(sfft, case):
    if case == "d1":
        sig, blocks = draw_signal(1, 4096, 40, seed=4), (1,)
    elif case == "d4_2x2":
        sig, blocks = draw_signal(4, 32, 60, seed=8), (2, 2)
    elif case == "d3_full_unwrap":
        sig, blocks = draw_signal(3, 64, 100, seed=5), (3,)
    elif case == "d6_tilted":
        sig, blocks = draw_signal(6, 128, 150, seed=6), (2, 2, 2)
    elif case == "signed_box":
        sig, blocks = draw_signal(3, 256, 80, seed=7, box_lo=-128), (2, 1)
    else:
        sig, blocks = draw_signal(12, 64, 120, seed=12), (3,) * 4
    dirs = None
    if case == "d6_tilted":
        dirs = [[1, 128, 7, 0, 0, 3], [0, 5, 1, 128, 0, 0], [11, 0, 0, 0, 1, 128]]
        blocks = None
    _assert_parity(sig, *_run_both(sfft, sig, blocks, dirs=dirs, box_lo=sig.box_lo), FP32_COEFF_TOL)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("residual", ["bins", "samples"])
def test_recovery_fp64_policy(sfft, residual, prec):
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = draw_signal(5, 1024, 300, seed=31, r_lo=1.0, r_hi=10.0)
    _assert_parity(sig, *_run_both(sfft, sig, wl.blocks, prec=prec, residual=residual),
                   FP64_COEFF_TOL if prec == "fp64" else DF64_COEFF_TOL)


def test_fig2_collision_story_on_gpu(sfft):
    w = np.array([[3, 5], [9, 5], [3, 12]])
    a = np.array([1.0 + 0.5j, -0.7 + 1.2j, 0.4 - 1.1j])
    from paper_1606_07407_gb300.inputs import Signal
    sig = Signal(2, 16, w.astype(np.int32), a)
    gf, ga, status, stats, ref = _run_both(sfft, sig, dirs=[[0, 1], [1, 0]], primes=[17])
    assert stats["accepted"][:2] == [1, 2]
    _assert_parity(sig, gf, ga, status, stats, ref, FP32_COEFF_TOL)


# ------------------------------------------------------------------ edge cases

def test_empty_signal(sfft):
    # nothing to find: one empty round per line direction (two blocks) under the float policy,
    # one under FP64
    s = sfft.Signal(np.zeros((0, 3), np.int32), np.zeros(0, np.complex128), 1024)
    for prec, rounds in (("fp32", 2), ("fp64", 1), ("df64", 1)):
        f, a, status, stats = sfft.Plan(3, 1024, 10, blocks=(2, 1), precision=prec).execute(s)
        assert status == 0 and f.shape[0] == 0 and stats["rounds"] == rounds


def test_single_mode(sfft):
    sig = draw_signal(4, 1 << 16, 1, seed=2)
    _assert_parity(sig, *_run_both(sfft, sig, (2, 2)), FP32_COEFF_TOL)


def test_capacity_overflow_reported(sfft):
    sig = draw_signal(2, 1024, 16, seed=1)
    plan = sfft.Plan(2, 1024, 16, blocks=(1, 1))
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, 1024), capacity=4, allow=(3,))
    assert status == 3 and f.shape[0] == 4


def test_not_converged_reported(sfft):
    # two modes that differ only in coordinate 2, projected on coordinate 1 every round, never separate
    w = np.array([[5, 10], [5, 11]], np.int32)
    a = np.array([1.0, 1.0j])
    plan = sfft.Plan(2, 1024, 2, dirs=[[1, 0]], max_rounds=6)
    f, _, status, stats = plan.execute(sfft.Signal(w, a, 1024), allow=(2,))
    assert status == 2 and stats["rounds"] == 6 and not stats["converged"]


def test_repeated_execute_is_stable(sfft):
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal()
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks)
    s = sfft.Signal(sig.freqs, sig.coeffs, sig.N)
    first = None
    for _ in range(3):
        f, a, status, _ = plan.execute(s)
        gf, ga = sfft.sort_result(_np(f), _np(a))
        if first is None:
            first = (gf, ga)
        assert status == 0 and np.array_equal(gf, first[0])
        assert np.max(np.abs(ga - first[1]) / np.abs(first[1])) < 1e-5


# ------------------------------------------------------------------ batches and graph mode

def _mixed_signals(n, seed):
    from paper_1606_07407_gb300.inputs import default_blocks
    st = Stream(seed)
    ks = st.integers(n, 8, 97)
    ds = st.integers(n, 2, 7)
    ls = st.integers(n, 10, 17)
    out = []
    for s in range(n):
        d, N, k = int(ds[s]), 1 << int(ls[s]), int(ks[s])
        out.append((draw_signal(d, N, k, seed=seed * 1000 + s, r_lo=1.0, r_hi=10.0), default_blocks(d, N, k)))
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_mixed_matches_oracle(sfft, graph):
    sigs = _mixed_signals(24, 44)
    plans = [sfft.Plan(s.d, s.N, s.k, blocks=b) for s, b in sigs]
    batch = sfft.Batch(plans, graph=graph)
    res, sts, stats = batch.execute([sfft.Signal(s.freqs, s.coeffs, s.N) for s, _ in sigs])
    assert all(x == 0 for x in sts)
    th = O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    for (sig, blocks), (f, a) in zip(sigs, res):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, blocks, th=th, estimator="mean")
        planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
        assert np.array_equal(gf, ref.freqs) and np.array_equal(gf, planted)
        assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL


def test_batch_equals_one_at_a_time(sfft):
    sigs = _mixed_signals(8, 45)
    plans = [sfft.Plan(s.d, s.N, s.k, blocks=b) for s, b in sigs]
    dev = [sfft.Signal(s.freqs, s.coeffs, s.N) for s, _ in sigs]
    res, sts, _ = sfft.Batch(plans).execute(dev)
    for plan, sg, (f, a) in zip(plans, dev, res):
        f1, a1, st1, _ = plan.execute(sg)
        g1 = sfft.sort_result(_np(f1), _np(a1))
        gb = sfft.sort_result(_np(f), _np(a))
        assert st1 == 0 and np.array_equal(g1[0], gb[0])
        # the mode splits of the sampling grid depend on the batch, so the float sums differ
        # in order: both are float estimates, compared at the float coefficient tolerance
        assert np.max(np.abs(g1[1] - gb[1]) / np.abs(g1[1])) < FP32_COEFF_TOL


def test_batch_of_d5_workload(sfft):
    wl = WORKLOADS["d5_N1024_k1000"]
    sigs = [wl.signal(seed_offset=s) for s in range(4)]
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks)
    res, sts, stats = sfft.Batch([plan] * 4, graph=True).execute(
        [sfft.Signal(s.freqs, s.coeffs, s.N) for s in sigs])
    assert sts == [0, 0, 0, 0]
    for sig, (f, a) in zip(sigs, res):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        order = np.lexsort(sig.freqs.T[::-1])
        assert np.array_equal(gf, sig.freqs[order])
        assert np.max(np.abs(ga - sig.coeffs[order]) / np.abs(sig.coeffs[order])) < FP32_COEFF_TOL


def test_graph_single_signal(sfft):
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=9)
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, graph=True)
    s = sfft.Signal(sig.freqs, sig.coeffs, sig.N)
    for _ in range(2):
        f, a, status, stats = plan.execute(s)
        gf, ga = sfft.sort_result(_np(f), _np(a))
        order = np.lexsort(sig.freqs.T[::-1])
        assert status == 0 and np.array_equal(gf, sig.freqs[order])


def test_paper_estimator_option(sfft):
    # coefficient a = Y_0[h] / p exactly as printed in Eq. 41, against the oracle with the same estimator
    wl = WORKLOADS["d2_N1024_k16"]
    sig = wl.signal(seed_offset=3)
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, coef="set0")
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, wl.blocks,
                             th=O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25), estimator="set0")
    _assert_parity(sig, gf, ga, status, stats, ref, FP32_COEFF_TOL)


def test_assign_many_refills_like_fresh_handles(sfft):
    # mixed d in one packed buffer; one handle refilled with fewer modes than it holds, one emptied
    sigs = _mixed_signals(6, 46)
    handles = [sfft.Signal(np.zeros((s.k, s.d), np.int32), np.zeros(s.k, np.complex128), s.N) for s, _ in sigs]
    ks = [s.k for s, _ in sigs]
    ks[2] -= 3
    ks[4] = 0
    fw = torch.tensor(np.concatenate([s.freqs[:k].reshape(-1) for (s, _), k in zip(sigs, ks)]).astype(np.int32),
                      device="cuda")
    ca = torch.tensor(np.concatenate([s.coeffs[:k] for (s, _), k in zip(sigs, ks)]), dtype=torch.complex128,
                      device="cuda")
    sfft.assign_many(handles, fw, ca, ks)
    for (sig, blocks), h, k in zip(sigs, handles, ks):
        plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=blocks)
        f, a, status, _ = plan.execute(h)
        f1, a1, status1, _ = plan.execute(sfft.Signal(sig.freqs[:k], sig.coeffs[:k], sig.N))
        assert h.k == k and status == 0 and status1 == 0
        g, g1 = sfft.sort_result(_np(f), _np(a)), sfft.sort_result(_np(f1), _np(a1))
        assert g[0].shape[0] == k and np.array_equal(g[0], g1[0])
        if k:
            assert np.max(np.abs(g[1] - g1[1]) / np.abs(g1[1])) < FP32_COEFF_TOL


# ------------------------------------------------------------------ noisy black boxes

def test_noisy_recovery_matches_oracle_noise_for_noise(sfft):
    # sigma = 0.01 moves the coefficients by a few 1e-5 relative (the noise of a bin over p), a
    # multiple of the float tolerance, so agreement with the oracle shows that both draw the
    # same noise for every sample
    d, N, k, sigma = 3, 256, 120, 1e-2
    sig = draw_signal(d, N, k, seed=43, r_lo=1.0, r_hi=10.0, noise_sigma=sigma)
    plan = sfft.Plan(d, N, k, blocks=(2, 1), tau=2e-2, noise_sigma=sigma, p_min=700)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, N, noise_sigma=sigma,
                                                   noise_seed=sig.noise_seed))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    th = O.Thresholds(tau=2e-2, rho=2.0 ** -17, delta=0.25, sigma=sigma)
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, (2, 1), th=th, estimator="mean", residual="bins",
                             noise=lambda i, p, dd: O.black_box_noise(sig.noise_seed, i, p, dd, sigma), p_min=700)
    order = np.lexsort(sig.freqs.T[::-1])
    assert status == 0 and ref.converged and min(stats["p"]) >= 700
    assert np.array_equal(gf, ref.freqs) and np.array_equal(gf, sig.freqs[order])
    assert stats["p"] == [r["p"] for r in ref.rounds]
    moved = np.abs(ref.coeffs - sig.coeffs[order]) / np.abs(sig.coeffs[order])
    assert np.median(moved) > 2 * FP32_COEFF_TOL                   # the noise is visible ...
    assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL   # ... and the same


def test_noisy_d10_workload_full_size(sfft):
    # d = 10, N = 2^16, k = 10^4, sigma = 1e-3 (FP64 phase ratio, four-step DFT), primes floored
    # at 30000 so that the read-out noise of |a| = 1 modes stays inside delta: the planted set,
    # and coefficient errors on the scale of the noise in a bin
    wl = WORKLOADS["d10_N65536_k10000_noisy"]
    sig = wl.signal()
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, noise_sigma=wl.noise_sigma, p_min=wl.p_min)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N, noise_sigma=wl.noise_sigma,
                                                   noise_seed=sig.noise_seed))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    order = np.lexsort(sig.freqs.T[::-1])
    assert status == 0 and stats["converged"]
    assert np.array_equal(gf, sig.freqs[order])
    err = np.abs(ga - sig.coeffs[order])
    ps, ns = stats["p"], wl.d + 1
    assert np.max(err) < 8 * wl.noise_sigma / math.sqrt(min(ps) * ns)
    assert np.sqrt(np.mean(err ** 2)) > 0.2 * wl.noise_sigma / math.sqrt(max(ps) * ns)


# ------------------------------------------------------------------ block shifts (Alg. 2 as printed)

@pytest.mark.parametrize("prec", ["fp32", "fp64", "df64"])
def test_block_shift_samples_match_oracle(sfft, prec):
    d, N, K, p, blocks = 5, 6, 300, 1031, (2, 3)
    sig = draw_signal(d, N, K, seed=71, r_lo=1.0, r_hi=10.0, box_lo=-3)
    plan = sfft.Plan(d, N, K, blocks=blocks, precision=prec, shift="block", box_lo=-3)
    assert plan.n_sets == 3
    u = [int(v) for v in O.unwrap_vector(d, N, blocks, 1)]
    y = _np(plan.sample(p, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs)))
    ref = O.sample_sets(sig.freqs, sig.coeffs, p, u, N, shift="block", blocks=blocks)
    assert y.shape == ref.shape and np.max(np.abs(y - ref)) < _sample_tol(prec, K, sig.coeffs)


@pytest.mark.parametrize("case", ["d6_auto", "d6_fp64", "paper_d100_fp64"])
def test_block_shift_recovery_matches_oracle(sfft, case):
    if case.startswith("d6"):
        d, N, k, blocks, box, unit, seed = 6, 16, 40, (3, 3), -8, False, 72
    else:
        d, N, k, blocks, box, unit, seed = 100, 20, 64, (5,) * 20, -10, True, 73
    prec = "fp64" if case.endswith("fp64") else "fp32"
    sig = draw_signal(d, N, k, seed=seed, box_lo=box, unit_modulus=unit, r_lo=1.0, r_hi=10.0)
    plan = sfft.Plan(d, N, k, blocks=blocks, precision=prec, shift="block", box_lo=box)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    th = O.Thresholds() if prec == "fp64" else O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, k, blocks, th=th, box_lo=box, estimator="mean",
                             residual="bins", shift="block", empty_rounds=FP64_EMPTY_ROUNDS if prec == "fp64" else None)
    _assert_parity(sig, gf, ga, status, stats, ref, FP64_COEFF_TOL if prec == "fp64" else FP32_COEFF_TOL)
    assert stats["samples"] == sum(r["samples"] for r in ref.rounds)


TILT_32 = (84, 13, 85)        # base, height, hypo: base > 2 N for N = 32 (Theorem 1)
TILT_1024 = (2112, 65, 2113)  # base > 2 N for N = 1024


@pytest.mark.parametrize("prec", ["fp32", "fp64", "df64"])
def test_tilt_samples_match_oracle(sfft, prec):
    N, K, p = 32, 300, 1031
    sig = draw_signal(2, N, K, seed=81, r_lo=1.0, r_hi=10.0)
    plan = sfft.Plan(2, N, K, precision=prec, shift="tilt", tilt=TILT_32)
    assert plan.n_sets == 3
    for u in O.tilt_axes(TILT_32):
        u = [int(v) for v in u]
        y = _np(plan.sample(p, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs)))
        ref = O.sample_sets(sig.freqs, sig.coeffs, p, u, N, shift="tilt", tilt=TILT_32)
        assert y.shape == ref.shape and np.max(np.abs(y - ref)) < _sample_tol(prec, K, sig.coeffs)


@pytest.mark.parametrize("case", ["N32_fp32", "N32_fp32_unfused", "N32_signed_fp32", "N1024_signed_fp64",
                                  "N1024_fp64_samples"])
def test_tilt_recovery_matches_oracle(sfft, case):
    # Alg. 3: lines along the rotated axes in turn, sets shifted along them by 1 / ((base + height) N),
    # read-out turned back; same sets, primes and coefficients as the oracle's tilted form
    if case.startswith("N32"):
        N, k, tilt, prec = 32, 40, TILT_32, "fp32"
    else:
        N, k, tilt, prec = 1024, 300, TILT_1024, "fp64"
    box = -N // 2 if "signed" in case else 0
    residual = "samples" if case.endswith("samples") else "bins"
    sig = draw_signal(2, N, k, seed=82 + len(case), box_lo=box, r_lo=1.0, r_hi=10.0)
    plan = sfft.Plan(2, N, k, precision=prec, shift="tilt", tilt=tilt, box_lo=box, residual=residual,
                     fuse="unfused" not in case)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    th = O.Thresholds() if prec == "fp64" else O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, 2, N, k, th=th, box_lo=box, estimator="mean",
                             residual=residual, shift="tilt", tilt=tilt,
                             empty_rounds=FP64_EMPTY_ROUNDS if prec == "fp64" else None)
    _assert_parity(sig, gf, ga, status, stats, ref, FP64_COEFF_TOL if prec == "fp64" else FP32_COEFF_TOL)
    assert stats["samples"] == sum(r["samples"] for r in ref.rounds)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tilt_resolves_rectangle_corners_that_parallel_projections_cannot(sfft, prec):
    # the worst case of Sec. 3.3: with lines along e_1 and e_2 every corner shares its bin with
    # another corner in every round (NOT_CONVERGED, nothing found); the tilted lines of Alg. 3
    # recover every corner (Theorem 1), as the oracle does
    N, tilt = (32, TILT_32) if prec == "fp32" else (1024, TILT_1024)
    sig = draw_rectangle_signal(N, 24, 6, seed=83)
    freqs, coeffs, k = sig.freqs, sig.coeffs, 24
    par = sfft.Plan(2, N, k, blocks=(1, 1), precision=prec, max_rounds=24)
    f, a, status, stats = par.execute(sfft.Signal(freqs, coeffs, N), allow=(0, 2))
    assert status == 2 and f.shape[0] < k
    plan = sfft.Plan(2, N, k, precision=prec, shift="tilt", tilt=tilt)
    f, a, status, stats = plan.execute(sfft.Signal(freqs, coeffs, N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    order = np.lexsort(freqs.T[::-1])
    assert status == 0 and np.array_equal(gf, freqs[order].astype(np.int64))
    th = O.Thresholds() if prec == "fp64" else O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    ref = O.multi_phaseshift(freqs, coeffs, 2, N, k, th=th, estimator="mean", residual="bins", shift="tilt",
                             tilt=tilt)
    assert np.array_equal(gf, ref.freqs)
    tol = FP64_COEFF_TOL if prec == "fp64" else FP32_COEFF_TOL
    assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < tol


def test_tilt_in_a_batch_with_other_forms(sfft):
    # per-slot shift forms: tilted, per-coordinate and block slots share the batched kernels
    N = 32
    specs = [("tilt", 2, None), ("coord", 2, (1, 1)), ("tilt", 2, None), ("block", 4, (2, 2))]
    sigs, plans, refs = [], [], []
    th = O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    for i, (shift, d, blocks) in enumerate(specs):
        sig = draw_signal(d, N, 24, seed=90 + i, r_lo=1.0, r_hi=10.0)
        kw = {"tilt": TILT_32} if shift == "tilt" else {"blocks": blocks}
        plans.append(sfft.Plan(d, N, 24, shift=shift, **kw))
        sigs.append(sig)
        refs.append(O.multi_phaseshift(sig.freqs, sig.coeffs, d, N, 24, blocks, th=th, estimator="mean",
                                       residual="bins", shift=shift, tilt=TILT_32 if shift == "tilt" else None))
    batch = sfft.Batch(plans)
    res, sts, stats = batch.execute([sfft.Signal(s.freqs, s.coeffs, N) for s in sigs])
    for (f, a), st, ref in zip(res, sts, refs):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        assert st == 0 and np.array_equal(gf, ref.freqs)
        assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL


def test_batch_beyond_one_plan_block_shares_tables_across_chunks(sfft):
    # more signals than the plan kernel's threads (its scans run in chunks of 256): sparsities
    # repeat across the chunks, so signals of one prime in different chunks share the tables
    # and filter of the first of them; every signal recovers its planted set, and a sample of
    # them matches the oracle coefficient by coefficient
    n, N = 320, 64
    ks = [8 + (t * 7) % 33 for t in range(n)]
    sigs = [draw_signal(2, N, k, seed=1200 + t, r_lo=1.0, r_hi=10.0) for t, k in enumerate(ks)]
    plans = {k: sfft.Plan(2, N, k, blocks=(2,)) for k in set(ks)}
    batch = sfft.Batch([plans[k] for k in ks])
    res, sts, stats = batch.execute([sfft.Signal(s.freqs, s.coeffs, N) for s in sigs])
    th = O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    for t, (s, (f, a), st) in enumerate(zip(sigs, res, sts)):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        order = np.lexsort(s.freqs.T[::-1])
        assert st == 0 and np.array_equal(gf, s.freqs[order].astype(np.int64))
        assert np.max(np.abs(ga - s.coeffs[order]) / np.abs(s.coeffs[order])) < 1e-4
        if t % 20 == 0:
            ref = O.multi_phaseshift(s.freqs, s.coeffs, 2, N, ks[t], (2,), th=th, estimator="mean", residual="bins")
            assert np.array_equal(gf, ref.freqs)
            assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL


@pytest.mark.parametrize("case", ["d2_blocks11", "d3_blocks21"])
def test_parallel_projection_failures_match_the_projection_core(sfft, case):
    # Sec. 2.2 / 4.2: the parallel projections never isolate the oracle's projection core; a batch
    # of random small signals recovers every other mode (FP64: exact set per signal) and stops
    # unconverged exactly where the core is not empty (float: the status per signal)
    d, N, k, blocks, n = (2, 16, 12, (1, 1), 96) if case == "d2_blocks11" else (3, 6, 24, (2, 1), 48)
    sigs = [draw_signal(d, N, k, seed=700 + t) for t in range(n)]
    cores = [set(O.projection_core(s.freqs, N, blocks).tolist()) for s in sigs]
    handles = [sfft.Signal(s.freqs, s.coeffs, N) for s in sigs]
    for prec in ("fp64", "fp32"):
        batch = sfft.Batch([sfft.Plan(d, N, k, blocks=blocks, precision=prec, max_rounds=40)] * n)
        res, sts, stats = batch.execute(handles, allow=(0, 2))
        for s, core, (f, a), st in zip(sigs, cores, res, sts):
            assert st == (2 if core else 0)
            if prec == "fp64":
                gf, ga = sfft.sort_result(_np(f), _np(a))
                keep = np.array([j for j in range(k) if j not in core], dtype=np.int64)
                want = s.freqs[keep][np.lexsort(s.freqs[keep].T[::-1])].astype(np.int64)
                wa = s.coeffs[keep][np.lexsort(s.freqs[keep].T[::-1])]
                assert np.array_equal(gf, want)
                assert np.max(np.abs(ga - wa) / np.abs(wa)) < 1e-9
    assert sum(bool(c) for c in cores) >= 3   # the batch includes failures


@pytest.mark.parametrize("d", [100, 1000])
def test_paper_experiment_exact_with_round_off_error(sfft, d):
    # Sec. 5: d = 100 and 1000, d1 = 5 (d2 = 20 and 200 blocks), N = 20, |a| = 1, box
    # [-N/2, N/2)^d, eps = 1 / (2 N^5): every frequency exact and the l2 coefficient error at
    # double round-off (the paper reports averages below 2^-52; a few ulps per mode here)
    for k, seed in ((1, 1), (32, 2), (1024, 3)):
        sig = draw_signal(d, 20, k, seed=seed * 100 + d, box_lo=-10, unit_modulus=True)
        plan = sfft.Plan(d, 20, k, blocks=(5,) * (d // 5), precision="fp64", shift="block", box_lo=-10)
        f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, 20))
        gf, ga = sfft.sort_result(_np(f), _np(a))
        order = np.lexsort(sig.freqs.T[::-1])
        assert status == 0 and np.array_equal(gf, sig.freqs[order])
        assert np.linalg.norm(ga - sig.coeffs[order]) < 16 * 2.0 ** -52 * math.sqrt(k) * 10


def test_precision_stress_d20_fp64_recovers_every_mode(sfft):
    # d = 20, N = 2^20, k = 10^5, |a| log-uniform in [1e-2, 1e2]: the all-FP64 policy reads every
    # mode (the float policies cannot: float sampling error over 10^5 modes with a 1e4 dynamic range
    # puts the small modes' phase read-out N Arg / (2 pi) far beyond delta at N = 2^20)
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = wl.signal()
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, precision="fp64")
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    order = np.lexsort(sig.freqs.T[::-1])
    assert status == 0 and np.array_equal(gf, sig.freqs[order])
    assert np.max(np.abs(ga - sig.coeffs[order]) / np.abs(sig.coeffs[order])) < 1e-9


# ------------------------------------------------------------------ stop rule over every set

@pytest.mark.parametrize("fuse", [True, False])
def test_stop_rule_reads_every_set(sfft, fuse):
    # a pair of opposite modes that lines along e_2 cannot separate: unconverged, not a wrong
    # set reported as converged (fused short rounds and batched kernels alike)
    from test_oracle_pins import _check_stop_rule

    def recover(w, a, N, dirs, max_rounds):
        plan = sfft.Plan(2, N, len(w), blocks=(1, 1), dirs=dirs, max_rounds=max_rounds, fuse=fuse)
        f, c, status, stats = plan.execute(sfft.Signal(w, a, N), allow=(0, 2))
        gf, ga = sfft.sort_result(_np(f), _np(c))
        assert (status == 0) == stats["converged"]
        return status == 0, gf, ga

    fa, ref = _check_stop_rule(recover)
    assert np.max(np.abs(fa - ref) / np.abs(ref)) < FP32_COEFF_TOL


# ------------------------------------------------------------------ the batched mix of independent signals

def _mix_slots_to_check(mix, n_check):
    """Slots spread over the mix's classes: the largest d, the largest N, the largest k, the
    smallest k (short lines, fused rounds), then evenly spaced others."""
    idx = [max(range(len(mix)), key=lambda i: (mix[i][0].d, mix[i][0].k)),
           max(range(len(mix)), key=lambda i: (mix[i][0].N, mix[i][0].k)),
           max(range(len(mix)), key=lambda i: mix[i][0].k),
           min(range(len(mix)), key=lambda i: mix[i][0].k)]
    step = max(1, len(mix) // max(1, n_check - len(idx)))
    for i in range(0, len(mix), step):
        if len(set(idx)) >= n_check:
            break
        idx.append(i)
    return sorted(set(idx))


def test_batched_mix_over_the_full_ranges_matches_oracle(sfft):
    # 256 signals with k ~ U{8..512}, d ~ U{2..8} (nine-set slots beside fused ones),
    # N = 2^U{10..20} (the double read-out above 2^14 beside the float one), each with the tuned
    # schedule of its class, one graph launch: every slot's set equals the planted one; sampled
    # slots equal the oracle's set (same schedule), with coefficients within the float tolerance
    from paper_1606_07407_gb300 import tuning
    from paper_1606_07407_gb300.inputs import BASE_SEED, batched_mix
    mix = batched_mix(256, seed=BASE_SEED + 4 + 77)
    assert {s.d for s, _ in mix} == set(range(2, 9))
    assert min(s.N for s, _ in mix) == 1 << 10 and max(s.N for s, _ in mix) == 1 << 20
    from paper_1606_07407_gb300.inputs import blocks_for
    sched = [tuning.schedule(s.d, s.N, s.k) for s, _ in mix]
    mix = [(s, blocks_for(s.d, s.N, s.k, sc["blocks"])) for (s, _), sc in zip(mix, sched)]
    plans = [sfft.Plan(s.d, s.N, s.k, blocks=b, c=sc["c"], p_min=sc["p_min"], fuse_max_len=sc["fuse_max_len"])
             for (s, b), sc in zip(mix, sched)]
    res, sts, stats = sfft.Batch(plans, graph=True).execute([sfft.Signal(s.freqs, s.coeffs, s.N) for s, _ in mix])
    assert sts == [0] * len(mix)
    got = []
    for (sig, _), (f, a) in zip(mix, res):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        assert np.array_equal(gf, sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64))
        got.append((gf, ga))
    th = O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25)
    for i in _mix_slots_to_check(mix, 10):
        sig, blocks = mix[i]
        ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, blocks, th=th, estimator="mean",
                                 residual="bins", c=sched[i]["c"], p_min=sched[i]["p_min"])
        assert ref.converged and np.array_equal(got[i][0], ref.freqs), i
        assert np.max(np.abs(got[i][1] - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL, i


def test_paper_estimator_at_the_d5_workload_size(sfft):
    # a = Y_0[h] / p exactly as printed in Eq. 41 on the d = 5, N = 1024, k = 1000 workload,
    # against the oracle with the same estimator: the same set and primes
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=11)
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, coef="set0")
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, wl.blocks,
                             th=O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25), estimator="set0",
                             residual="bins")
    planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
    assert status == 0 and ref.converged
    assert np.array_equal(gf, ref.freqs) and np.array_equal(gf, planted)
    rel = np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)
    print(f"Eq. 41 estimator at d = 5, k = 1000: max rel err {rel.max():.3e}, median {np.median(rel):.3e}")
    # one set's bin carries its own float rounding; the default estimator averages the d + 1 sets'
    # independent roundings (within 1e-5), so the one-set estimate is held to sqrt(d + 1) times that
    # (measured: max 1.1e-5, median 2.2e-7)
    assert rel.max() < FP32_COEFF_TOL * math.sqrt(sig.d + 1)


@pytest.mark.parametrize("fuse", [True, False])
def test_stop_rule_waits_for_every_line_direction(sfft, fuse):
    # a +-1 pair one unit apart at N = 2^20 that only the third block's line separates: the float
    # policy recovers all three modes (fused short rounds and batched kernels alike)
    from test_oracle_pins import _check_every_direction_stop

    def recover(w, a, N):
        plan = sfft.Plan(3, N, len(w), blocks=(1, 1, 1), fuse=fuse)
        f, c, status, stats = plan.execute(sfft.Signal(w, a, N), allow=(0, 2))
        gf, ga = sfft.sort_result(_np(f), _np(c))
        return status == 0, gf, ga

    fa, ref = _check_every_direction_stop(recover)
    assert np.max(np.abs(fa - ref) / np.abs(ref)) < FP32_COEFF_TOL


# ------------------------------------------------------------------ dense split-BF16 tensor-core DFT

DENSE_FLUSH = 4      # K tiles (32 samples each) per tensor-memory accumulation segment


def _split_bf16_dft_tol(p, y, Y=None):
    # Each operand is split into two BF16 terms, hi = bf16(v) and lo = bf16(v - hi): 8 significant
    # bits each, so v - hi - lo is below 2^-16 |v| (two round-to-nearest steps of 2^-8), and the
    # dropped lo_A lo_B is below 2^-16 |A| |B|.  Each of the 2p real products of a bin carries
    # about 3 2^-16 |A| |B| with |A| <= 1, and these add like a random walk: six standard
    # deviations of it per row.  The tensor core rounds each MMA's sum into its FP32 accumulator
    # (12 MMAs per tile, up to 2^-23 of the partial sum each); where the products add coherently
    # those roundings add up, so the kernel drains the accumulator into registers every
    # DENSE_FLUSH tiles: at most 12 DENSE_FLUSH 2^-23 |Y| from the segments, plus a 2^-24 |Y| per
    # register addition (one per segment).
    rms = np.sqrt(np.mean(np.abs(y) ** 2, axis=1, keepdims=True))
    walk = 6.0 * 3 * 2.0 ** -16 * math.sqrt(2 * p) * rms
    seg = 12 * DENSE_FLUSH * 2.0 ** -23 + math.ceil(p / (32 * DENSE_FLUSH)) * 2.0 ** -24
    mag = np.abs(Y) if Y is not None else 0.0
    return walk + seg * (mag + 6.0 * math.sqrt(64 * DENSE_FLUSH) * rms)


@pytest.mark.parametrize("p", [2, 5, 83, 911, 2039, 4099, 8191])
def test_dense_bf16_dft_matches_definition(sfft, p):
    # kernel (b) on the tensor cores (tcgen05, split BF16, FP32 accumulate) for primes up to 8191,
    # against the DFT by its definition (Eq. 3) in FP64, every bin of every set
    d = 5
    plan = sfft.Plan(d, 1024, 2000, precision="fp32_bf16dft")
    rng = np.random.default_rng(p)
    y = (rng.standard_normal((d + 1, p)) + 1j * rng.standard_normal((d + 1, p))) * np.array([[1.0], [0.5], [2], [1],
                                                                                              [3], [0.25]])
    Y = _np(plan.dft(p, torch.tensor(y.astype(np.complex64), device="cuda")))
    ref = O.dft(y.astype(np.complex64).astype(np.complex128))
    err = np.abs(Y - ref)
    assert np.all(err <= _split_bf16_dft_tol(p, y, ref)), float(err.max())
    # and the error is split-BF16 sized, not plain BF16 (8 bits: about 2^-8 of each product)
    rms = np.sqrt(np.mean(np.abs(y) ** 2))
    if p >= 83:
        assert err.max() < 2.0 ** -11 * math.sqrt(2 * p) * rms


def test_dense_bf16_dft_single_mode_closed_form(sfft):
    # one mode: Y_0 is p a at bin (w . u) mod p and zero elsewhere, to the split-BF16 error
    d, N, p = 3, 4096, 4099
    w = np.array([[1234, 77, 3000]], np.int32)
    a = np.array([1.5 - 0.5j])
    plan = sfft.Plan(d, N, 1000, precision="fp32_bf16dft", blocks=(3,))   # primes up to about 5000
    u = [int(v) for v in O.unwrap_vector(d, N, (3,), 0)]
    y = plan.sample(p, u, torch.tensor(w, device="cuda"), torch.tensor(a, device="cuda"))
    Y = _np(plan.dft(p, y))
    h = int(sum(int(x) * int(v) for x, v in zip(w[0], u)) % p)
    yc = _np(y).astype(np.complex128)
    peak = np.zeros((1, p))
    peak[0, h] = p * abs(a[0])
    tol = _split_bf16_dft_tol(p, yc[:1], peak)
    assert abs(Y[0, h] - p * a[0]) <= tol[0, h]
    Y[0, h] = 0
    assert np.all(np.abs(Y[0]) <= tol[0])


def test_recovery_with_the_dense_bf16_dft_matches_oracle(sfft):
    # the d = 5, N = 1024, k = 1000 workload with every round's DFT on the tensor cores (its primes
    # are all below 8191): the same set as the oracle; the coefficients carry the split-BF16 DFT's
    # error, about 3 2^-16 sqrt(2 / p) |y|_rms / |a| relative, reported here
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=21)
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, precision="fp32_bf16dft")
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, wl.blocks,
                             th=O.Thresholds(tau=1e-3, rho=2.0 ** -17, delta=0.25), estimator="mean",
                             residual="bins")
    planted = sig.freqs[np.lexsort(sig.freqs.T[::-1])].astype(np.int64)
    assert status == 0 and np.array_equal(gf, ref.freqs) and np.array_equal(gf, planted)
    assert stats["launches"]["fused"] == 0 and all(p <= 8191 for p in stats["p"])
    rel = np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)
    yrms = math.sqrt(float(np.sum(np.abs(sig.coeffs) ** 2)))
    bound = (6 * 3 * 2.0 ** -16 * math.sqrt(2.0 / min(stats["p"])) * yrms
             + (12 * DENSE_FLUSH * 2.0 ** -23) * np.abs(ref.coeffs)) / np.abs(ref.coeffs)
    print(f"split-BF16 DFT recovery: max rel coefficient error {rel.max():.3e}, median {np.median(rel):.3e}")
    assert np.all(rel < bound)


# ------------------------------------------------------------------ float rounds, then double rounds

def test_float_then_double_recovers_the_precision_stress_shape(sfft):
    # d = 20, N = 2^20, |a| log-uniform in [1e-2, 1e2], k = 1000: float rounds alone read only the
    # modes of |a| >~ 1 and stall (about 40% found); the policy hands the float registry to double
    # rounds, which find the rest and cancel float false positives: the planted set exactly, the
    # coefficients of the float-found modes within the float tolerance, the others at double's
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = draw_signal(wl.d, wl.N, 1000, wl.seed + 100, wl.r_dist, wl.r_lo, wl.r_hi)
    plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, precision="fp32_then_fp64")
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    order = np.lexsort(sig.freqs.T[::-1])
    assert status == 0 and np.array_equal(gf, sig.freqs[order].astype(np.int64))
    assert np.max(np.abs(ga - sig.coeffs[order]) / np.abs(sig.coeffs[order])) < FP32_COEFF_TOL
    ref = O.multi_phaseshift(sig.freqs, sig.coeffs, sig.d, sig.N, sig.k, wl.blocks, residual="bins", estimator="mean")
    assert np.array_equal(gf, ref.freqs)
    assert np.max(np.abs(ga - ref.coeffs) / np.abs(ref.coeffs)) < FP32_COEFF_TOL
    fp32 = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, precision="fp32", max_rounds=24)
    f32, _, st32, _ = fp32.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N), allow=(2,))
    assert st32 == 2 and f32.shape[0] < sig.k           # float alone does not recover it
    # the double rounds continue the round counter: their primes are new ones
    assert len(stats["p"]) == stats["rounds"] and all(p > 0 for p in stats["p"])


def test_float_then_double_equals_float_where_float_suffices(sfft):
    # the d = 5 workload converges in the float rounds: the policy returns their result (the same
    # set and primes; coefficients to the float tolerance, since float atomics add in any order)
    wl = WORKLOADS["d5_N1024_k1000"]
    sig = wl.signal(seed_offset=31)
    got = []
    for prec in ("fp32", "fp32_then_fp64"):
        plan = sfft.Plan(sig.d, sig.N, sig.k, blocks=wl.blocks, precision=prec)
        f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
        assert status == 0
        got.append((sfft.sort_result(_np(f), _np(a)), stats["p"]))
    assert np.array_equal(got[0][0][0], got[1][0][0])
    assert np.max(np.abs(got[0][0][1] - got[1][0][1]) / np.abs(got[0][0][1])) < FP32_COEFF_TOL
    assert got[0][1] == got[1][1]


def test_float_then_double_is_refused_in_a_batch(sfft):
    plan = sfft.Plan(2, 1024, 16, precision="fp32_then_fp64")
    with pytest.raises(sfft.SfftError) as err:
        sfft.Batch([plan])
    assert err.value.status == 1


# ------------------------------------------------------------------ double-float sampling

def test_double_float_samples_at_the_precision_stress_size(sfft):
    # d = 20, N = 2^20, K = 100000 modes of |a| log-uniform in [1e-2, 1e2], the first prime of the
    # workload's schedule: 48 sampled columns of all 21 sets against the oracle, within the
    # double-float bound, and at least 2^16 times closer than float sampling's bound
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = wl.signal()
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, precision="df64")
    p = 500009
    u = [int(v) for v in O.unwrap_vector(wl.d, wl.N, wl.blocks, 3)]
    y = _np(plan.sample(p, u, torch.tensor(sig.freqs), torch.tensor(sig.coeffs)))
    xs = np.array(sorted(set(Stream(9).integers(46, 0, p).tolist()) | {0, p - 1}))
    ref = O.sample_sets(sig.freqs, sig.coeffs, p, u, wl.N, x_values=xs)
    err = np.max(np.abs(y[:, xs] - ref))
    print(f"double-float samples, K = 1e5: max |err| {err:.3e}, sum |a| {np.sum(np.abs(sig.coeffs)):.3e}")
    assert err < _df64_sample_tol(wl.k, sig.coeffs)
    assert err < 2.0 ** -16 * _sample_tol("fp32", wl.k, sig.coeffs)


def test_double_float_recovers_the_precision_stress_shape(sfft):
    # the d = 20, N = 2^20 log-uniform shape at k = 1000, where the float policies stall: the
    # planted set exactly, the oracle's rounds and primes, coefficients within DF64_COEFF_TOL of the
    # oracle's
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = draw_signal(wl.d, wl.N, 1000, wl.seed + 100, wl.r_dist, wl.r_lo, wl.r_hi)
    _assert_parity(sig, *_run_both(sfft, sig, wl.blocks, prec="df64"), DF64_COEFF_TOL)


def test_precision_stress_d20_df64_recovers_every_mode(sfft):
    # the full d = 20 precision-stress workload (k = 10^5) under double-float sampling: every
    # planted mode, coefficients within 1e-9 relative of the planted values (as FP64)
    wl = WORKLOADS["d20_N1048576_k100000"]
    sig = wl.signal()
    plan = sfft.Plan(wl.d, wl.N, wl.k, blocks=wl.blocks, precision="df64", graph=True)
    f, a, status, stats = plan.execute(sfft.Signal(sig.freqs, sig.coeffs, sig.N))
    gf, ga = sfft.sort_result(_np(f), _np(a))
    order = np.lexsort(sig.freqs.T[::-1])
    assert status == 0 and np.array_equal(gf, sig.freqs[order])
    rel = np.abs(ga - sig.coeffs[order]) / np.abs(sig.coeffs[order])
    print(f"df64 d20 k=1e5: rounds {stats['rounds']}, max rel coefficient error {rel.max():.3e}")
    assert np.max(rel) < 1e-9


def test_double_float_batch_matches_one_at_a_time_and_refuses_fp64(sfft):
    sigs = [draw_signal(4, 1 << 12, 60 + 20 * s, seed=900 + s, r_lo=1.0, r_hi=10.0) for s in range(3)]
    plans = [sfft.Plan(s.d, s.N, s.k, blocks=(2, 2), precision="df64") for s in sigs]
    res, sts, _ = sfft.Batch(plans).execute([sfft.Signal(s.freqs, s.coeffs, s.N) for s in sigs])
    for s, (f, a), st in zip(sigs, res, sts):
        gf, ga = sfft.sort_result(_np(f), _np(a))
        order = np.lexsort(s.freqs.T[::-1])
        assert st == 0 and np.array_equal(gf, s.freqs[order])
        assert np.max(np.abs(ga - s.coeffs[order]) / np.abs(s.coeffs[order])) < DF64_COEFF_TOL
    with pytest.raises(sfft.SfftError) as err:
        sfft.Batch([plans[0], sfft.Plan(4, 1 << 12, 60, blocks=(2, 2), precision="fp64")])
    assert err.value.status == 1
