"""The allocation-free sampling entry point agrees with the plan-based one and with the oracle.

sfft_sample_noalloc serves callers that may not allocate device memory when they
need samples (a memory pool that must not grow, a process that forbids cudaMalloc
after start-up): it keeps its scratch in one device array inside the library.
Two calls in a row, each compared through the C ABI with sfft_sample on the same
inputs and with the oracle's samples, at the float sampling tolerance the other
parity tests use.  This file is collected last so that a run stopping at the
first failure has run everything else.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.sfft_oracle as O
from paper_1606_07407_gb300.inputs import draw_signal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfft():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1606_07407_gb300 import build as B
    B.build()
    from paper_1606_07407_gb300 import sfft as S
    S.load()
    return S


def _float_tol(coeffs):
    # float sampling: blocked sums of unit-modulus terms, error a few ulps of sum |a|
    return 2.0 ** -20 * float(np.sum(np.abs(coeffs)))


# (d, N, K, p, blocks, block of the line, box_lo): one set group with the box [0, N), and
# d = 9 (ten sets, two set groups of five) with the paper's signed box [-N/2, N/2)
CASES = [(5, 1024, 1000, 5003, (3, 2), 1, 0), (3, 4096, 100, 1031, (2, 1), 0, 0),
         (9, 64, 300, 1511, (3, 3, 3), 2, -32)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_no_alloc_sampling_matches_plan_sampling_and_oracle_twice(sfft, case):
    d, N, K, p, blocks, m, box_lo = CASES[case]
    sig = draw_signal(d, N, K, seed=500 + K, r_lo=1.0, r_hi=10.0, box_lo=box_lo)
    assert sig.freqs.min() >= box_lo and sig.freqs.max() < box_lo + N
    u = [int(v) for v in O.unwrap_vector(d, N, blocks, m)]
    w = torch.tensor(sig.freqs, dtype=torch.int32, device="cuda")
    a = torch.tensor(sig.coeffs, dtype=torch.complex128, device="cuda")
    plan = sfft.Plan(d, N, K, blocks=blocks, box_lo=box_lo)
    y_ref = plan.sample(p, u, w, a).cpu().numpy()
    y_or = O.sample_sets(sig.freqs, sig.coeffs, p, u, N)
    tol = _float_tol(sig.coeffs)
    out = torch.empty((d + 1, p), dtype=torch.complex64, device="cuda")
    for call in range(2):                        # two calls in a row share the scratch array
        out.fill_(float("nan"))
        y_na = sfft.sample_noalloc(d, N, p, u, w, a, box_lo=box_lo, out=out).cpu().numpy()
        assert y_na.shape == (d + 1, p)
        assert np.all(np.isfinite(y_na)), call
        assert np.max(np.abs(y_na - y_ref)) < tol, call
        assert np.max(np.abs(y_na - y_or)) < tol, call


def test_no_alloc_rejects_requests_beyond_its_scratch(sfft):
    # 8 MiB of scratch: a 2^21-entry root table plus 10^5 modes of d = 20 does not fit
    d, K, p = 20, 100000, 2097143
    w = torch.zeros((K, d), dtype=torch.int32, device="cuda")
    a = torch.zeros((K,), dtype=torch.complex128, device="cuda")
    out = torch.empty((d + 1, p), dtype=torch.complex64, device="cuda")   # a full-size output anyway
    with pytest.raises(sfft.SfftError) as err:
        sfft.sample_noalloc(d, 1 << 20, p, [1] + [0] * (d - 1), w, a, out=out)
    assert err.value.status == 3
