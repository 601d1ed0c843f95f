"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1606_07407_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sfft_plan_create", "sfft_execute", "sfft_signal_synthetic", "sfft_sample", "sfft_dft",
                 "sfft_classify", "sfft_plan_destroy", "sfft_signal_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_knows_every_declared_symbol():
    from paper_1606_07407_gb300 import sfft
    assert sorted(sfft.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib):
    lib.sfft_status_string.restype = ctypes.c_char_p
    assert lib.sfft_status_string(0) == b"ok"
    assert lib.sfft_status_string(2) == b"not converged"


def test_invalid_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sfft_plan_create(0, ctypes.c_int64(16), ctypes.c_int64(4), None, None, None, None,
                                ctypes.byref(h)) == 1
    assert lib.sfft_plan_create(2, ctypes.c_int64(1), ctypes.c_int64(4), None, None, None, None,
                                ctypes.byref(h)) == 1
    assert lib.sfft_execute(None, None, ctypes.c_int64(0), None, None, None, None) == 1
    assert lib.sfft_signal_assign_many(-1, None, None, None, None, None) == 1
    handles = (ctypes.c_void_p * 2)(None, None)
    ks = (ctypes.c_int64 * 2)(3, 4)
    assert lib.sfft_signal_assign_many(2, handles, ks, None, None, None) == 1
    assert lib.sfft_signal_assign_many(0, None, None, None, None, None) == 0   # nothing to do
    from paper_1606_07407_gb300.sfft import _Opts
    bad = _Opts(0, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 7, 0)                       # unknown residual form
    assert lib.sfft_plan_create(2, ctypes.c_int64(16), ctypes.c_int64(4), None, None, ctypes.byref(bad), None,
                                ctypes.byref(h)) == 1
    # block shifts read N^{d1} values from one phase: beyond 2^20 only the FP64 policy may (PRECISION = 4)
    from paper_1606_07407_gb300.sfft import _Tilts
    blk = (ctypes.c_int * 20)(*([5] * 20))
    tl = _Tilts(0, None, 20, blk)
    block = _Opts(0, -10, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 0, 1)
    assert lib.sfft_plan_create(100, ctypes.c_int64(20), ctypes.c_int64(16), None, ctypes.byref(tl),
                                ctypes.byref(block), None, ctypes.byref(h)) == 4
    assert lib.sfft_plan_sets(None) == -1


def test_more_plan_arguments_rejected_without_gpu(lib):
    # every check of sfft_plan_create runs before the engine touches the device
    from paper_1606_07407_gb300.sfft import _Opts, _PSchedule, _Tilts
    h = ctypes.c_void_p()

    def create(d=2, N=64, k=8, ps=None, tl=None, **opt):
        o = _Opts(0, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 0, 0)
        for key, v in opt.items():
            setattr(o, key, v)
        return lib.sfft_plan_create(d, ctypes.c_int64(N), ctypes.c_int64(k), ctypes.byref(ps) if ps else None,
                                    ctypes.byref(tl) if tl else None, ctypes.byref(o), None, ctypes.byref(h))

    assert create(shift=3) == 1                       # unknown shift form
    assert create(precision=9) == 1                   # unknown precision policy
    assert create(box_lo=1) == 1                      # the box starts at most at 0
    assert create(delta=0.5) == 1                     # read-out tolerance below half an integer
    assert create(max_rounds=-1) == 1
    assert create(N=1 << 24) == 4                     # a float policy reads N values from a phase
    primes = (ctypes.c_int64 * 2)(101, 91)            # 91 = 7 * 13
    assert create(ps=_PSchedule(0, 2, primes, 0)) == 1
    assert create(ps=_PSchedule(0, 0, None, 1 << 27)) == 1   # prime floor beyond the tables
    blocks = (ctypes.c_int * 2)(2, 2)                 # block sizes must add up to d
    assert create(tl=_Tilts(0, None, 2, blocks)) == 1


def test_tilt_arguments_rejected_without_gpu(lib):
    # the tilted form (Alg. 3) takes d = 2 and a primitive Pythagorean triple; its read-out
    # resolves Q = (base + height) N values, beyond 2^21 under a float policy only in FP64
    from paper_1606_07407_gb300.sfft import _Opts
    h = ctypes.c_void_p()

    def create(d, N, triple, precision=0):
        o = _Opts(precision, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 0, 2)
        o.tilt_base, o.tilt_height, o.tilt_hypo = triple
        return lib.sfft_plan_create(d, ctypes.c_int64(N), ctypes.c_int64(8), None, None, ctypes.byref(o), None,
                                    ctypes.byref(h))

    assert create(3, 32, (84, 13, 85)) == 1          # not two-dimensional
    assert create(2, 32, (84, 13, 86)) == 1          # not Pythagorean
    assert create(2, 32, (8, 6, 10)) == 1            # not primitive
    assert create(2, 32, (0, 1, 1)) == 1             # a leg of zero
    assert create(2, 1024, (2112, 65, 2113), precision=1) == 4   # Q = 2.2e6 > 2^21 in float (PRECISION)


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_batch_results_slice_each_signal_from_the_flat_outputs():
    torch = pytest.importorskip("torch")
    from paper_1606_07407_gb300.sfft import BatchResults
    d, caps, found = [2, 3, 1], [4, 2, 5], [3, 7, 0]      # the second signal overflowed its capacity
    fo = torch.arange(sum(c * k for c, k in zip(caps, d)), dtype=torch.int32)
    co = torch.arange(sum(caps), dtype=torch.float64).to(torch.complex128)
    res = BatchResults(d, caps, fo, co, found)
    assert len(res) == 3
    f0, a0 = res[0]
    assert f0.shape == (3, 2) and f0.flatten().tolist() == list(range(6)) and a0.real.tolist() == [0, 1, 2]
    f1, a1 = res[1]
    assert f1.shape == (2, 3) and f1.flatten().tolist() == list(range(8, 14)) and a1.real.tolist() == [4, 5]
    f2, a2 = res[-1]
    assert f2.shape == (0, 1) and a2.numel() == 0
    assert [f.shape[0] for f, _ in res] == [3, 2, 0] and len(res[1:]) == 2
    with pytest.raises(IndexError):
        res[3]


def test_sampling_wrappers_reject_bad_shapes_before_any_device_call(monkeypatch):
    # the kernels read K d frequencies and K coefficients and write (d + 1) p samples: a tensor
    # of another shape or dtype would be read or written out of bounds, so the binding refuses it
    # before it loads the library or touches the device
    torch = pytest.importorskip("torch")
    from paper_1606_07407_gb300 import sfft as S

    def no_device(*_a, **_k):
        raise AssertionError("reached the library")

    monkeypatch.setattr(S, "load", no_device)
    w = torch.zeros((10, 3), dtype=torch.int32)
    a = torch.zeros((10,), dtype=torch.complex128)
    u = [1, 0, 0]
    with pytest.raises(ValueError):
        S.sample_noalloc(4, 64, 11, [1, 0, 0, 0], w, a)                  # freqs not [K, d]
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, u, w, a[:5])                         # K coefficients expected
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, u, w.reshape(-1), a)                 # freqs not two-dimensional
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, u, w, a, out=torch.empty((4, 10), dtype=torch.complex64))   # too short
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, u, w, a, out=torch.empty((3, 11), dtype=torch.complex64))   # too few sets
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, u, w, a, out=torch.empty((4, 11), dtype=torch.complex128))  # wrong dtype
    with pytest.raises(ValueError):
        S.sample_noalloc(3, 64, 11, [1, 0], w, a)                        # direction of d entries
    # the plan-based step wrappers check the same things before their calls
    plan = S.Plan.__new__(S.Plan)
    plan.d = 3
    with pytest.raises(ValueError):
        plan.sample(11, u, torch.zeros((10, 2), dtype=torch.int32), a)
    with pytest.raises(ValueError):
        plan.sample(11, u, w, a[:3])


def test_assign_many_rejects_mismatched_counts_before_any_device_call(monkeypatch):
    # one mode count per handle: a short or long ks list would make the library read past an array
    torch = pytest.importorskip("torch")
    from paper_1606_07407_gb300 import sfft as S

    def no_device(*_a, **_k):
        raise AssertionError("reached the library")

    monkeypatch.setattr(S, "load", no_device)

    class Handle:
        def __init__(self):
            self._h = ctypes.c_void_p(None)
            self.k = 0

    sigs = [Handle(), Handle()]
    w = torch.zeros((7, 2), dtype=torch.int32)
    a = torch.zeros((7,), dtype=torch.complex128)
    with pytest.raises(ValueError):
        S.assign_many(sigs, w, a, [3])
    with pytest.raises(ValueError):
        S.assign_many(sigs, w, a, [3, 2, 2])


def test_precision_policy_range_without_gpu(lib):
    # the policies are AUTO .. DF64 (0 .. 6); anything else is refused before any CUDA call
    from paper_1606_07407_gb300.sfft import PREC, _Opts
    assert PREC["df64"] == 6 and PREC["fp32_then_fp64"] == 5 and PREC["fp32_bf16dft"] == 4
    h = ctypes.c_void_p()
    for prec in (-1, 7):
        bad = _Opts(prec, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0, 0, 0)
        assert lib.sfft_plan_create(2, ctypes.c_int64(16), ctypes.c_int64(4), None, None, ctypes.byref(bad), None,
                                    ctypes.byref(h)) == 1


def test_double_float_cost_model_of_the_bench():
    # (4 products x 12 operations per set, plus 32 for E shared by the group's sets) / 2 samples
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert abs(bench.df64_ops_per_term(20) - (48 + 32 / 7) / 2) < 1e-12    # 21 sets: 3 groups of 7
    assert abs(bench.df64_ops_per_term(4) - (48 + 32 / 5) / 2) < 1e-12     # 5 sets: one group
    assert abs(bench.df64_ops_per_term(8) - (48 + 32 / 5) / 2) < 1e-12     # 9 sets: 2 groups of 5


def test_precision_study_rejects_unknown_arms_before_any_device_work():
    from paper_1606_07407_gb300 import precision_study as P
    with pytest.raises(SystemExit):
        P.main(["--arms", "fp64,bogus"])
