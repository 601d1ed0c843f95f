"""Python binding of the C ABI in include/sfft.h (argument marshalling only).

Every call goes to libsfft.so; nothing here computes any step of the method.
Device buffers are torch CUDA tensors; the plan runs on torch's current CUDA
stream unless another stream is given.  Import fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

PREC = {"fp32": 0, "auto": 0, "fp32_fp64ratio": 1, "fp32_only": 2, "fp64": 3, "fp32_bf16dft": 4,
        "fp32_then_fp64": 5, "df64": 6}
STATUS = {0: "ok", 1: "invalid argument", 2: "not converged", 3: "capacity exceeded",
          4: "beyond phase resolution", 5: "more modes than k", 6: "cuda error", 7: "device wait timed out"}
MAX_ROUNDS = 256
NKCLASS = 7
KCLASSES = ("setup", "project", "sample", "dft", "classify", "merge", "fused")


class SfftError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class _PSchedule(C.Structure):
    _fields_ = [("c_prime", C.c_int), ("n_primes", C.c_int), ("primes", C.POINTER(C.c_int64)),
                ("p_min", C.c_int64), ("c_eighths", C.c_int)]


def prime_factor_eighths(c) -> int:
    """The prime factor c of the rule p >= c k* in eighths (the ABI's c_eighths); c must be a
    multiple of 1/8 in [1/8, 4096] so that ceil(c k*) is exact on every side."""
    c8 = round(float(c) * 8)
    if abs(float(c) * 8 - c8) > 1e-9 or not 1 <= c8 <= 8 * 4096:
        raise ValueError(f"prime factor c = {c} is not a multiple of 1/8 in [1/8, 4096]")
    return int(c8)


class _Tilts(C.Structure):
    _fields_ = [("n_dirs", C.c_int), ("dirs", C.POINTER(C.c_int64)), ("n_blocks", C.c_int),
                ("block_sizes", C.POINTER(C.c_int))]


# where g (the registry's function) leaves f: its transform subtracted bin by bin, or its
# samples subtracted at every sample point
RESIDUAL = {"bins": 0, "samples": 1}
# shifted sets: one per coordinate (e_n / N), one per unwrapping block (Alg. 2 as printed), or
# one per rotated axis of the tilted lines (Alg. 3, d = 2)
SHIFT = {"coord": 0, "block": 1, "tilt": 2}


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("box_lo", C.c_int), ("tau", C.c_double), ("rho", C.c_double),
                ("delta", C.c_double), ("noise_sigma", C.c_double), ("max_rounds", C.c_int),
                ("profile", C.c_int), ("graph", C.c_int), ("coef_set0", C.c_int), ("residual", C.c_int),
                ("shift", C.c_int), ("unfused", C.c_int),
                ("tilt_base", C.c_int), ("tilt_height", C.c_int), ("tilt_hypo", C.c_int),
                ("fuse_max_len", C.c_int), ("empty_rounds", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("rounds", C.c_int), ("converged", C.c_int), ("samples", C.c_int64), ("terms", C.c_int64),
                ("terms_fused", C.c_int64),
                ("p", C.c_int64 * MAX_ROUNDS), ("K", C.c_int32 * MAX_ROUNDS),
                ("accepted", C.c_int32 * MAX_ROUNDS), ("registry", C.c_int32 * MAX_ROUNDS),
                ("kernel_launches", C.c_int64 * NKCLASS), ("kernel_ms", C.c_double * NKCLASS)]


EXPORTS = ["sfft_plan_create", "sfft_plan_destroy", "sfft_signal_synthetic", "sfft_signal_destroy",
           "sfft_signal_assign", "sfft_signal_assign_many",
           "sfft_execute", "sfft_batch_create", "sfft_batch_destroy", "sfft_batch_device_bytes",
           "sfft_batch_execute", "sfft_sample", "sfft_sample_noalloc", "sfft_dft", "sfft_classify",
           "sfft_plan_max_prime",
           "sfft_plan_mode_capacity", "sfft_plan_sets", "sfft_plan_device_bytes", "sfft_last_cuda_error",
           "sfft_status_string"]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> C.CDLL:
    """Loads libsfft.so (built by paper_1606_07407_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libsfft.so not built ({path}); run paper_1606_07407_gb300.build.build()")
    L = C.CDLL(path)
    vp, i64, i32p, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)
    L.sfft_plan_create.argtypes = [C.c_int, i64, i64, C.POINTER(_PSchedule), C.POINTER(_Tilts), C.POINTER(_Opts),
                                   vp, C.POINTER(vp)]
    L.sfft_plan_create.restype = C.c_int
    L.sfft_plan_destroy.argtypes = [vp]
    L.sfft_plan_destroy.restype = None
    L.sfft_signal_synthetic.argtypes = [C.c_int, i64, i64, vp, vp, C.c_double, C.c_uint64, C.POINTER(vp)]
    L.sfft_signal_synthetic.restype = C.c_int
    L.sfft_signal_destroy.argtypes = [vp]
    L.sfft_signal_destroy.restype = None
    L.sfft_signal_assign.argtypes = [vp, i64, vp, vp]
    L.sfft_signal_assign.restype = C.c_int
    L.sfft_signal_assign_many.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(i64), vp, vp, vp]
    L.sfft_signal_assign_many.restype = C.c_int
    L.sfft_execute.argtypes = [vp, vp, i64, vp, vp, C.POINTER(i64), C.POINTER(_Stats)]
    L.sfft_execute.restype = C.c_int
    L.sfft_batch_create.argtypes = [C.c_int, C.POINTER(vp), vp, C.c_int, C.POINTER(vp)]
    L.sfft_batch_create.restype = C.c_int
    L.sfft_batch_destroy.argtypes = [vp]
    L.sfft_batch_destroy.restype = None
    L.sfft_batch_device_bytes.argtypes = [vp]
    L.sfft_batch_device_bytes.restype = i64
    L.sfft_batch_execute.argtypes = [vp, C.POINTER(vp), C.POINTER(i64), vp, vp, C.POINTER(i64),
                                     C.POINTER(C.c_int32), C.POINTER(_Stats)]
    L.sfft_batch_execute.restype = C.c_int
    L.sfft_sample.argtypes = [vp, i64, C.POINTER(i64), i64, vp, vp, vp]
    L.sfft_sample.restype = C.c_int
    L.sfft_sample_noalloc.argtypes = [C.c_int, i64, i64, C.POINTER(i64), i64, vp, vp, vp, C.c_int, vp]
    L.sfft_sample_noalloc.restype = C.c_int
    L.sfft_dft.argtypes = [vp, i64, C.c_int, vp, vp]
    L.sfft_dft.restype = C.c_int
    L.sfft_classify.argtypes = [vp, i64, C.POINTER(i64), vp, C.c_double, i64, vp, vp, vp, C.POINTER(i64)]
    L.sfft_classify.restype = C.c_int
    for f in ("sfft_plan_max_prime", "sfft_plan_mode_capacity", "sfft_plan_device_bytes"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = i64
    L.sfft_plan_sets.argtypes = [vp]
    L.sfft_plan_sets.restype = C.c_int
    L.sfft_last_cuda_error.argtypes = []
    L.sfft_last_cuda_error.restype = C.c_int
    L.sfft_status_string.argtypes = [C.c_int]
    L.sfft_status_string.restype = C.c_char_p
    _lib = L
    return L


def _check(st: int, what: str, ok=(0,)):
    if st not in ok:
        if st == 6:
            what += f" (cudaError {load().sfft_last_cuda_error()})"
        raise SfftError(st, what)
    return st


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _i64_array(vals):
    arr = (C.c_int64 * len(vals))(*[int(v) for v in vals])
    return arr


class Signal:
    """Synthetic black box f(t) = sum_j coeffs_j e^{2 pi i freqs_j . t} held on the device; with
    noise_sigma > 0 every sample carries complex Gaussian noise drawn from noise_seed."""

    def __init__(self, freqs, coeffs, N: int, noise_sigma: float = 0.0, noise_seed: int = 0):
        L = load()
        freqs = torch.as_tensor(np.asarray(freqs) if not torch.is_tensor(freqs) else freqs)
        coeffs = torch.as_tensor(np.asarray(coeffs) if not torch.is_tensor(coeffs) else coeffs)
        self.k, self.d = int(freqs.shape[0]), int(freqs.shape[1])
        self.N = int(N)
        fw = freqs.to(device="cuda", dtype=torch.int32).contiguous()
        ca = coeffs.to(device="cuda", dtype=torch.complex128).contiguous()
        h = C.c_void_p()
        self.noise_sigma, self.noise_seed = float(noise_sigma), int(noise_seed)
        _check(L.sfft_signal_synthetic(self.d, self.N, self.k, _ptr(fw), _ptr(ca), self.noise_sigma,
                                       self.noise_seed & 0xFFFFFFFFFFFFFFFF, C.byref(h)), "sfft_signal_synthetic")
        self._h = h

    def assign(self, freqs: torch.Tensor, coeffs: torch.Tensor):
        """Replaces the modes in place (device tensors int32 [k, d] and complex128 [k])."""
        _check(load().sfft_signal_assign(self._h, int(freqs.shape[0]), _ptr(freqs), _ptr(coeffs)),
               "sfft_signal_assign")
        self.k = int(freqs.shape[0])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sfft_signal_destroy(h)
            self._h = None


def assign_many(signals, freqs: torch.Tensor, coeffs: torch.Tensor, ks, stream=None):
    """Refills the handles from packed device tensors: signal s takes ks[s] modes, its rows of
    freqs (int32 [sum ks, d]) and entries of coeffs (complex128 [sum ks]) following those of the
    signals before it.  Enqueued on the stream (default: torch's current one), not waited for."""
    n = len(signals)
    karr = np.ascontiguousarray(ks, dtype=np.int64)
    if karr.shape != (n,):
        raise ValueError("ks must have one entry per signal")
    if stream is None:
        stream = torch.cuda.current_stream()
    harr = np.fromiter((s._h.value for s in signals), dtype=np.uint64, count=n)
    _check(load().sfft_signal_assign_many(n, harr.ctypes.data_as(C.POINTER(C.c_void_p)),
                                          karr.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(freqs), _ptr(coeffs),
                                          C.c_void_p(stream.cuda_stream)),
           "sfft_signal_assign_many")
    for s, k in zip(signals, ks):
        s.k = int(k)


class Plan:
    """An sfft plan: d, N, k, prime schedule, line directions and precision policy."""

    def __init__(self, d: int, N: int, k: int, blocks=None, dirs=None, primes=None, c: float = 5,
                 precision: str = "fp32", box_lo: int = 0, tau: float = 0.0, rho: float = 0.0,
                 delta: float = 0.0, noise_sigma: float = 0.0, max_rounds: int = 0, stream=None,
                 profile: bool = False, graph: bool = False, coef: str = "mean", residual: str = "bins",
                 p_min: int = 0, shift: str = "coord", fuse: bool = True, tilt=None, fuse_max_len: int = 0,
                 empty_rounds: int = 0):
        L = load()
        if residual not in RESIDUAL:
            raise ValueError(f"residual must be one of {sorted(RESIDUAL)}")
        self.d, self.N, self.k = int(d), int(N), int(k)
        self.precision = precision
        self.cdtype = torch.complex128 if precision in ("fp64", "df64") else torch.complex64
        self._keep = []
        ps = _PSchedule(0, 0, None, int(p_min), prime_factor_eighths(c))
        if primes is not None and len(primes):
            arr = _i64_array(primes)
            self._keep.append(arr)
            ps.n_primes, ps.primes = len(primes), arr
        tl = _Tilts(0, None, 0, None)
        if dirs is not None and len(dirs):
            flat = [int(v) for row in dirs for v in row]
            arr = _i64_array(flat)
            self._keep.append(arr)
            tl.n_dirs, tl.dirs = len(dirs), arr
        elif blocks is not None:
            arr = (C.c_int * len(blocks))(*[int(b) for b in blocks])
            self._keep.append(arr)
            tl.n_blocks, tl.block_sizes = len(blocks), arr
        op = _Opts(PREC[precision], int(box_lo), float(tau), float(rho), float(delta), float(noise_sigma),
                   int(max_rounds), 1 if profile else 0, 1 if graph else 0, 1 if coef == "set0" else 0,
                   RESIDUAL[residual], SHIFT[shift], 0 if fuse else 1)
        op.fuse_max_len = int(fuse_max_len)
        op.empty_rounds = int(empty_rounds)
        if tilt is not None:   # (base, height, hypo) of the tilted form
            op.tilt_base, op.tilt_height, op.tilt_hypo = (int(v) for v in tilt)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(L.sfft_plan_create(self.d, self.N, self.k, C.byref(ps), C.byref(tl), C.byref(op),
                                  C.c_void_p(stream.cuda_stream), C.byref(h)), "sfft_plan_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sfft_plan_destroy(h)
            self._h = None

    @property
    def n_sets(self) -> int:
        """Sample sets per round: d + 1 (coordinate shifts) or 1 + blocks (block shifts)."""
        return int(load().sfft_plan_sets(self._h))

    @property
    def max_prime(self) -> int:
        return int(load().sfft_plan_max_prime(self._h))

    @property
    def device_bytes(self) -> int:
        return int(load().sfft_plan_device_bytes(self._h))

    def execute(self, signal: Signal, capacity: int | None = None, out=None, allow=(0,)):
        """Runs Algorithm 2; returns (freqs int32 [n, d], coeffs complex128 [n], status, stats) on the device."""
        L = load()
        cap = int(capacity if capacity is not None else max(2 * self.k + 16, 16))
        if out is None:
            fo = torch.empty((cap, self.d), dtype=torch.int32, device="cuda")
            co = torch.empty((cap,), dtype=torch.complex128, device="cuda")
        else:
            fo, co = out
        n = C.c_int64(0)
        st = _Stats()
        status = L.sfft_execute(self._h, signal._h, cap, _ptr(fo), _ptr(co), C.byref(n), C.byref(st))
        _check(status, "sfft_execute", ok=allow)
        m = min(int(n.value), cap)
        return fo[:m], co[:m], status, _stats_dict(st)

    def sample(self, p: int, u, freqs: torch.Tensor, coeffs: torch.Tensor) -> torch.Tensor:
        check_mode_arrays(self.d, torch.as_tensor(freqs), torch.as_tensor(coeffs))
        if len(u) != self.d:
            raise ValueError(f"u must have {self.d} entries")
        L = load()
        fw = freqs.to(device="cuda", dtype=torch.int32).contiguous()
        ca = coeffs.to(device="cuda", dtype=torch.complex128).contiguous()
        y = torch.empty((self.n_sets, int(p)), dtype=self.cdtype, device="cuda")
        ua = _i64_array(u)
        _check(L.sfft_sample(self._h, int(p), ua, int(fw.shape[0]), _ptr(fw), _ptr(ca), _ptr(y)), "sfft_sample")
        return y

    def dft(self, p: int, y: torch.Tensor) -> torch.Tensor:
        if y.dim() != 2 or int(y.shape[1]) != int(p) or not 1 <= int(y.shape[0]) <= self.n_sets:
            raise ValueError(f"y must be [rows <= {self.n_sets}, {int(p)}], got {tuple(y.shape)}")
        L = load()
        y = y.to(device="cuda", dtype=self.cdtype).contiguous()
        Y = torch.empty_like(y)
        _check(L.sfft_dft(self._h, int(p), int(y.shape[0]), _ptr(y), _ptr(Y)), "sfft_dft")
        return Y

    def classify(self, p: int, u, Y: torch.Tensor, eta_bin: float, capacity: int | None = None):
        if tuple(Y.shape) != (self.n_sets, int(p)) or len(u) != self.d:
            raise ValueError(f"Y must be [{self.n_sets}, {int(p)}] and u of {self.d} entries")
        L = load()
        Y = Y.to(device="cuda", dtype=self.cdtype).contiguous()
        cap = int(capacity if capacity is not None else p)
        h = torch.empty((max(cap, 1),), dtype=torch.int32, device="cuda")
        w = torch.empty((max(cap, 1), self.d), dtype=torch.int32, device="cuda")
        a = torch.empty((max(cap, 1),), dtype=torch.complex128, device="cuda")
        n = C.c_int64(0)
        ua = _i64_array(u)
        _check(L.sfft_classify(self._h, int(p), ua, _ptr(Y), float(eta_bin), cap, _ptr(h), _ptr(w), _ptr(a),
                               C.byref(n)), "sfft_classify")
        m = int(n.value)
        return h[:m], w[:m], a[:m]


def check_mode_arrays(d: int, freqs, coeffs) -> int:
    """Raises ValueError unless freqs is [K, d] and coeffs holds K entries; returns K.  The
    kernels read K d frequencies and K coefficients, so a mismatch would read out of bounds."""
    if freqs.dim() != 2 or int(freqs.shape[1]) != int(d):
        raise ValueError(f"freqs must be [K, {d}], got {tuple(freqs.shape)}")
    if coeffs.dim() != 1 or int(coeffs.shape[0]) != int(freqs.shape[0]):
        raise ValueError(f"coeffs must hold {int(freqs.shape[0])} entries, got {tuple(coeffs.shape)}")
    return int(freqs.shape[0])


def check_samples_out(out, d: int, p: int, dtype) -> None:
    """Raises ValueError unless `out` is a contiguous [d + 1, p] tensor of `dtype` (the kernel
    writes (d + 1) p samples)."""
    if out.dtype != dtype or tuple(out.shape) != (int(d) + 1, int(p)) or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {dtype} tensor of shape ({int(d) + 1}, {int(p)}), "
                         f"got {out.dtype} {tuple(out.shape)}")


def sample_noalloc(d: int, N: int, p: int, u, freqs: torch.Tensor, coeffs: torch.Tensor, box_lo: int = 0,
                   stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Samples of kernel (a) through the allocation-free entry point (the library allocates
    nothing; `out`, if given, receives the complex64 [d+1, p] samples).  Shapes and dtypes are
    checked before any device call.  Waits for the stream."""
    freqs, coeffs = torch.as_tensor(freqs), torch.as_tensor(coeffs)
    check_mode_arrays(d, freqs, coeffs)
    if out is not None:
        check_samples_out(out, d, p, torch.complex64)
    if len(u) != int(d):
        raise ValueError(f"u must have {d} entries")
    L = load()
    fw = freqs.to(device="cuda", dtype=torch.int32).contiguous()
    ca = coeffs.to(device="cuda", dtype=torch.complex128).contiguous()
    y = out if out is not None else torch.empty((d + 1, int(p)), dtype=torch.complex64, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream()
    ua = _i64_array(u)
    _check(L.sfft_sample_noalloc(int(d), int(N), int(p), ua, int(fw.shape[0]), _ptr(fw), _ptr(ca), _ptr(y),
                                 int(box_lo), C.c_void_p(stream.cuda_stream)), "sfft_sample_noalloc")
    stream.synchronize()
    return y


def _stats_dict(st: _Stats) -> dict:
    r = min(st.rounds, MAX_ROUNDS)
    return {"rounds": st.rounds, "converged": bool(st.converged), "samples": int(st.samples),
            "terms": int(st.terms), "terms_fused": int(st.terms_fused), "p": list(st.p[:r]), "K": list(st.K[:r]),
            "accepted": list(st.accepted[:r]), "registry": list(st.registry[:r]),
            "launches": dict(zip(KCLASSES, list(st.kernel_launches))),
            "kernel_ms": dict(zip(KCLASSES, list(st.kernel_ms)))}


class Batch:
    """Many independent signals recovered together: every kernel launch serves all slots."""

    def __init__(self, plans, stream=None, graph: bool = False, profile: bool = False):
        L = load()
        self.plans = list(plans)
        self.n = len(self.plans)
        arr = (C.c_void_p * self.n)(*[p._h.value for p in self.plans])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        flags = (1 if graph else 0) | (2 if profile else 0)
        _check(L.sfft_batch_create(self.n, arr, C.c_void_p(stream.cuda_stream), flags, C.byref(h)),
               "sfft_batch_create")
        self._h = h
        self.d = [p.d for p in self.plans]
        self.k = [p.k for p in self.plans]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sfft_batch_destroy(h)
            self._h = None

    @property
    def device_bytes(self) -> int:
        return int(load().sfft_batch_device_bytes(self._h))

    def outputs(self, caps=None):
        caps = [2 * k + 16 for k in self.k] if caps is None else [int(c) for c in caps]
        fo = torch.empty((sum(c * d for c, d in zip(caps, self.d)),), dtype=torch.int32, device="cuda")
        co = torch.empty((sum(caps),), dtype=torch.complex128, device="cuda")
        return caps, fo, co

    def execute(self, signals, out=None, allow=(0,)):
        """Returns (results, statuses, stats); results[s] is (freqs [n_s, d_s], coeffs [n_s]) as
        device tensors, sliced from the flat outputs when it is indexed."""
        L = load()
        caps, fo, co = out if out is not None else self.outputs()
        handles = tuple(s._h.value for s in signals)
        if handles != getattr(self, "_sig_key", None):       # the handle array is kept between calls
            self._sig_key = handles
            self._sig_arr = (C.c_void_p * self.n)(*handles)
        if getattr(self, "_caps_key", None) != tuple(caps):
            self._caps_key = tuple(caps)
            self._caps_arr = (C.c_int64 * self.n)(*caps)
        nf = (C.c_int64 * self.n)()
        sts = (C.c_int32 * self.n)()
        st = _Stats()
        status = L.sfft_batch_execute(self._h, self._sig_arr, self._caps_arr, _ptr(fo), _ptr(co), nf, sts,
                                      C.byref(st))
        _check(status, "sfft_batch_execute", ok=allow)
        return BatchResults(self.d, caps, fo, co, list(nf)), list(sts), _stats_dict(st)


class BatchResults:
    """Per-signal results of one batched execution.  Building hundreds of tensor views costs
    milliseconds of host time, so an entry is sliced from the flat outputs only when asked for."""

    def __init__(self, d, caps, fo, co, n_found):
        self.n_found = n_found
        self._d, self._fo, self._co = d, fo, co
        self._caps = caps
        self._r0 = self._e0 = None

    def __len__(self):
        return len(self._caps)

    def __getitem__(self, s):
        if isinstance(s, slice):
            return [self[i] for i in range(*s.indices(len(self)))]
        if s < 0:
            s += len(self)
        if not 0 <= s < len(self):
            raise IndexError(s)
        if self._r0 is None:
            self._r0 = np.concatenate([[0], np.cumsum(self._caps)]).tolist()
            self._e0 = np.concatenate([[0], np.cumsum([c * d for c, d in zip(self._caps, self._d)])]).tolist()
        m = min(int(self.n_found[s]), self._caps[s])
        r0, e0, d = self._r0[s], self._e0[s], self._d[s]
        return self._fo[e0:e0 + m * d].view(m, d), self._co[r0:r0 + m]

    def __iter__(self):
        for s in range(len(self)):
            yield self[s]


def sort_result(freqs: np.ndarray, coeffs: np.ndarray):
    """Lexicographic order of the frequency vectors (the result is a set)."""
    freqs = np.asarray(freqs)
    if freqs.shape[0] == 0:
        return freqs.astype(np.int64), np.asarray(coeffs)
    order = np.lexsort(freqs.T[::-1])
    return freqs[order].astype(np.int64), np.asarray(coeffs)[order]
