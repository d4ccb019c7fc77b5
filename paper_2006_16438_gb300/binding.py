"""Thin Python binding of the C ABI in include/cpa.h (libcpa.so).

Argument marshalling only: every step of the computation runs in the CUDA library.
Device buffers are torch CUDA tensors; torch supplies memory and the stream.  There
is no CPU fallback: if the library or a CUDA device is missing, calls raise.

The function names follow the C ABI: ``cpa_index_build``, ``cp_arls_lev``,
``cpa_skrp_lev``, ``cpa_sampled_mttkrp``, ...
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from . import _build

OK = 0
ERR_ARG = -1
ERR_COO_RANGE = -2
ERR_COO_DUP = -3
ERR_OOM = -4
ERR_REJECT_LIMIT = -5
ERR_DET_CAP = -6
ERR_CUDA = -7
ERR_UNSUPPORTED = -8
WARN_SINGULAR_GRAM = 1
WARN_RANK_DEFICIENT_LEV = 2
F32 = 1
F64 = 2
FP64 = 0
MIXED = 1
DIST_LEVERAGE = 0
DIST_UNIFORM = 1
DIST_LENGTH_SQUARED = 2
FIT_NONE = 0
FIT_EXACT = 1
FIT_ESTIMATED = 2

EXPORTED = [
    "cpa_options_default", "cpa_strerror", "cpa_index_build", "cpa_index_free", "cpa_index_info",
    "cpa_index_export", "cp_arls_lev", "cp_arls_lev_coo", "cpa_philox4x64", "cpa_leverage",
    "cpa_cdf", "cpa_skrp_lev", "cpa_sampled_mttkrp", "cpa_solve", "cpa_fit", "cpa_leverage_noalloc",
    "cpa_mode_update", "cp_als", "cpa_batch_create", "cpa_batch_run", "cpa_batch_info", "cpa_batch_free",
    "cpa_fit_sample", "cpa_fit_estimate", "cpa_rrf_init", "cpa_index_device_bytes", "cpa_fit_terms",
]


class CpaError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = _lib().cpa_strerror(code).decode() if _handle is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


class Coo(C.Structure):
    _fields_ = [("order", C.c_int32), ("dims", C.c_void_p), ("nnz", C.c_int64), ("idx", C.c_void_p),
                ("vals", C.c_void_p), ("val_dtype", C.c_int32), ("on_device", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("rank", C.c_int32), ("samples", C.c_int64), ("tau", C.c_double), ("iters", C.c_int32),
                ("epoch_len", C.c_int32), ("patience", C.c_int32), ("tol", C.c_double),
                ("seed", C.c_uint64), ("iter_offset", C.c_uint64), ("precision", C.c_int32),
                ("distribution", C.c_int32), ("fit_mode", C.c_int32), ("fit_samples", C.c_int64), ("fit_alpha", C.c_double),
                ("det_cap", C.c_int64), ("reject_cap", C.c_int32),
                ("profile", C.c_int32), ("stream", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("mode_updates", C.c_int32), ("warnings", C.c_int32),
                ("epochs", C.c_int32), ("sdet_last", C.c_int64), ("sbar_last", C.c_int64),
                ("nnz_sampled_last", C.c_int64), ("attempts_last", C.c_int64),
                ("pdet_last", C.c_double), ("nnz_sampled_total", C.c_int64),
                ("sbar_total", C.c_int64), ("stage_ms", C.c_double * 12),
                ("stage_launches", C.c_int64 * 12), ("kernel_launches", C.c_int64)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k in ("stage_ms", "stage_launches") else v
        return out


_handle = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcpa.so (building it with nvcc if it is missing or stale)."""
    global _handle
    if _handle is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcpa.so not found at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        _declare(lib)
        _handle = lib
    return _handle


def _lib():
    return load()


def _declare(lib):
    P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "cpa_options_default": ([P], None),
        "cpa_strerror": ([I32], C.c_char_p),
        "cpa_index_build": ([P, P, P], I32),
        "cpa_index_free": ([P], I32),
        "cpa_index_info": ([P, I32, P, P, P, P], I32),
        "cpa_index_device_bytes": ([P, P], I32),
        "cpa_index_export": ([P, I32, P, P, P, P, P], I32),
        "cp_arls_lev": ([P, P, P, P, I32, P, P], I32),
        "cp_arls_lev_coo": ([P, P, P, P, I32, P, P], I32),
        "cp_als": ([P, P, P, P, I32, P, P], I32),
        "cpa_batch_create": ([I32, P, P, P, P, P, I32, P, P], I32),
        "cpa_batch_run": ([P, P, P], I32),
        "cpa_batch_info": ([P, P, P, P, P], I32),
        "cpa_batch_free": ([P], I32),
        "cpa_mode_update": ([P, P, I32, U64, P, P, P, P, P, P, P], I32),
        "cpa_philox4x64": ([P, P, I64, P, P], I32),
        "cpa_leverage": ([P, I64, I32, P, P], I32),
        "cpa_leverage_noalloc": ([P, I64, I32, P, P], I32),
        "cpa_cdf": ([P, I64, I32, P, P, P], I32),
        "cpa_skrp_lev": ([I32, P, P, I32, P, I32, U64, P, P, P, P, P], I32),
        "cpa_sampled_mttkrp": ([P, I32, P, I32, P, P, I64, P, P, P, P], I32),
        "cpa_solve": ([P, P, I64, I32, P, P, P], I32),
        "cpa_fit": ([P, P, P, I32, P, P], I32),
        "cpa_fit_terms": ([P, P, P, I32, P, P], I32),
        "cpa_fit_sample": ([P, I64, D, U64, I32, P, P, P, P, P], I32),
        "cpa_rrf_init": ([P, I32, I64, U64, P, I32, P, P], I32),
        "cpa_fit_estimate": ([P, P, P, P, P, I64, P, P, I32, I32, P, P, P], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the CP-ARLS-LEV library needs a CUDA device; none is available")
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc, where):
    if rc < 0:
        raise CpaError(rc, where)
    return rc


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _ptr_array(ptrs):
    return (C.c_void_p * len(ptrs))(*ptrs)


def default_options(**kw) -> Options:
    o = Options()
    _lib().cpa_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# --------------------------------------------------------------------------- index
class Index:
    """A tensor index built by cpa_index_build; frees itself."""

    def __init__(self, handle, dims, nnz, val_dtype):
        self.h = handle
        self.dims = tuple(dims)
        self.nnz = nnz
        self.val_dtype = val_dtype

    @property
    def order(self):
        return len(self.dims)

    def nfib(self, k):
        n = C.c_int64(0)
        _check(_lib().cpa_index_info(self.h, k, None, None, None, C.byref(n)), "cpa_index_info")
        return n.value

    def device_bytes(self):
        """Device memory the index holds (bytes)."""
        n = C.c_int64(0)
        _check(_lib().cpa_index_device_bytes(self.h, C.byref(n)), "cpa_index_device_bytes")
        return n.value

    def free(self):
        if self.h is not None and self.h.value:
            _lib().cpa_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _coo_struct(dims, idx_ptrs, vals_ptr, nnz, val_dtype, on_device):
    d = np.asarray(dims, dtype=np.int64)
    ip = _ptr_array(idx_ptrs)
    s = Coo(len(dims), d.ctypes.data, int(nnz), C.cast(ip, C.c_void_p).value, vals_ptr, val_dtype,
            1 if on_device else 0)
    s._keep = (d, ip)
    return s


def coo_from_host(coo, dtype=np.float64):
    """cpa_coo over host numpy arrays of a synth.Coo-like object (kept alive on the
    returned struct)."""
    idx = [np.ascontiguousarray(i, dtype=np.int32) for i in coo.idx]
    vals = np.ascontiguousarray(coo.vals, dtype=dtype)
    s = _coo_struct(coo.dims, [i.ctypes.data for i in idx], vals.ctypes.data, vals.shape[0],
                    F32 if dtype == np.float32 else F64, False)
    s._arrays = (idx, vals)
    return s


def coo_from_device(dims, idx_tensors, vals_tensor):
    torch = _torch()
    dt = F32 if vals_tensor.dtype == torch.float32 else F64
    s = _coo_struct(dims, [t.data_ptr() for t in idx_tensors], vals_tensor.data_ptr(),
                    vals_tensor.shape[0], dt, True)
    s._arrays = (idx_tensors, vals_tensor)
    return s


def cpa_index_build(coo, dtype=np.float64, device_tensors=None) -> Index:
    """Build the per-mode fibre index.  ``coo``: a synth.Coo (host arrays), or
    ``device_tensors=(idx_list, vals)`` of CUDA tensors."""
    _torch()
    if device_tensors is not None:
        s = coo_from_device(coo.dims if hasattr(coo, "dims") else coo, *device_tensors)
        dims = coo.dims if hasattr(coo, "dims") else coo
    else:
        s = coo_from_host(coo, dtype)
        dims = coo.dims
    h = C.c_void_p(0)
    _check(_lib().cpa_index_build(C.byref(s), _stream(), C.byref(h)), "cpa_index_build")
    return Index(h, dims, s.nnz, s.val_dtype)


def cpa_index_export(index: Index, k: int):
    """Device copy of the fibre index of mode k: (keys, off, ik, val) CUDA tensors."""
    torch = _torch()
    F = index.nfib(k)
    keys = torch.empty(max(F, 1), dtype=torch.uint64, device="cuda")
    off = torch.empty(F + 1, dtype=torch.uint64, device="cuda")
    ik = torch.empty(max(index.nnz, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(index.nnz, 1), dtype=torch.float32 if index.val_dtype == F32 else torch.float64,
                      device="cuda")
    _check(_lib().cpa_index_export(index.h, k, _ptr(keys), _ptr(off), _ptr(ik), _ptr(val), _stream()),
           "cpa_index_export")
    return keys[:F], off, ik[:index.nnz], val[:index.nnz]


# --------------------------------------------------------------------------- driver
@dataclass
class Result:
    lam: object
    factors: list
    fit: float
    stats: dict
    warnings: int


def cp_arls_lev(index: Index, factors, *, rank, samples, tau=1.0, iters=10, epoch_len=5, patience=3,
                tol=0.0, seed=0, iter_offset=0, fit_mode=FIT_EXACT, det_cap=1 << 24,
                reject_cap=4096, on_device=True, profile=0, out=None, precision=FP64,
                fit_samples=1 << 27, fit_alpha=0.5, distribution=DIST_LEVERAGE, inplace=False) -> Result:
    """Alg. 3 on the GPU.  ``factors``: list of CUDA float64 tensors (n_k x rank), or
    numpy arrays with on_device=False (host buffers: the library copies them in and
    the results out).  Returns a Result with new factor copies; with on_device=False
    and inplace=True the caller's arrays (C-contiguous float64, e.g. views of pinned
    memory) receive the results instead."""
    torch = _torch()
    o = default_options(rank=rank, samples=int(samples), tau=float(tau), iters=int(iters),
                        epoch_len=int(epoch_len), patience=int(patience), tol=float(tol),
                        seed=int(seed), iter_offset=int(iter_offset), fit_mode=int(fit_mode),
                        det_cap=int(det_cap), reject_cap=int(reject_cap), profile=int(profile),
                        precision=int(precision), fit_samples=int(fit_samples), fit_alpha=float(fit_alpha),
                        distribution=int(distribution))
    o.stream = _stream()
    stats = Stats()
    fit = C.c_double(0.0)
    if on_device:
        if out is not None:  # caller-owned device buffers, updated in place
            fs, lam, fit_d = out
        else:
            fs = [f.detach().to(device="cuda", dtype=torch.float64).contiguous().clone() for f in factors]
            lam = torch.empty(rank, dtype=torch.float64, device="cuda")
            fit_d = torch.empty(1, dtype=torch.float64, device="cuda")
        rc = _lib().cp_arls_lev(index.h, C.byref(o), _ptr(lam), _ptr_array([f.data_ptr() for f in fs]), 1,
                                _ptr(fit_d), C.byref(stats))
        _check(rc, "cp_arls_lev")
        return Result(lam, fs, float(fit_d.item()), stats.as_dict(), rc)
    if inplace:
        fs = list(factors)
        if not all(isinstance(f, np.ndarray) and f.dtype == np.float64 and f.flags.c_contiguous for f in fs):
            raise ValueError("inplace factors must be C-contiguous float64 numpy arrays")
    else:
        fs = [np.ascontiguousarray(f, dtype=np.float64).copy() for f in factors]
    lam = np.zeros(rank)
    rc = _lib().cp_arls_lev(index.h, C.byref(o), lam.ctypes.data, _ptr_array([f.ctypes.data for f in fs]),
                            0, C.byref(fit), C.byref(stats))
    _check(rc, "cp_arls_lev")
    return Result(lam, fs, fit.value, stats.as_dict(), rc)


def cp_als(index: Index, factors, *, rank, iters=10, fit_mode=FIT_EXACT, precision=FP64) -> Result:
    """Full CP-ALS on the GPU (exact MTTKRP).  ``factors``: CUDA float64 tensors
    (n_k x rank); returns a Result with new factor copies."""
    torch = _torch()
    o = default_options(rank=rank, iters=int(iters), fit_mode=int(fit_mode), precision=int(precision))
    o.stream = _stream()
    stats = Stats()
    fs = [f.detach().to(device="cuda", dtype=torch.float64).contiguous().clone() for f in factors]
    lam = torch.empty(rank, dtype=torch.float64, device="cuda")
    fit_d = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = _lib().cp_als(index.h, C.byref(o), _ptr(lam), _ptr_array([f.data_ptr() for f in fs]), 1,
                       _ptr(fit_d), C.byref(stats))
    _check(rc, "cp_als")
    return Result(lam, fs, float(fit_d.item()), stats.as_dict(), rc)


class Batch:
    """Many fixed-length cp_arls_lev calls replayed as one CUDA graph (cpa_batch_*).
    problems: list of dicts with keys index, factors (CUDA float64 tensors), rank,
    samples, tau, iters, seed and optionally precision, iter_offset.  The factors are
    updated in place by every run()."""

    def __init__(self, problems, autotune=True):
        torch = _torch()
        self.problems = problems
        n = len(problems)
        self.lams = [torch.empty(p["rank"], dtype=torch.float64, device="cuda") for p in problems]
        self.fits_d = [torch.empty(1, dtype=torch.float64, device="cuda") for p in problems]
        self.factors = [p["factors"] for p in problems]
        opts = (Options * n)()
        for i, p in enumerate(problems):
            opts[i] = default_options(rank=p["rank"], samples=int(p["samples"]), tau=float(p["tau"]),
                                      iters=int(p["iters"]), seed=int(p.get("seed", 0)),
                                      iter_offset=int(p.get("iter_offset", 0)),
                                      precision=int(p.get("precision", FP64)),
                                      fit_mode=int(p.get("fit_mode", FIT_EXACT)),
                                      distribution=int(p.get("distribution", DIST_LEVERAGE)),
                                      fit_samples=int(p.get("fit_samples", 1 << 27)),
                                      fit_alpha=float(p.get("fit_alpha", 0.5)), stream=_stream())
        self._fac_arrays = [_ptr_array([f.data_ptr() for f in fs]) for fs in self.factors]
        fac_ptrs = (C.c_void_p * n)(*[C.cast(a, C.c_void_p) for a in self._fac_arrays])
        idx = (C.c_void_p * n)(*[p["index"].h.value for p in problems])
        lam_ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in self.lams])
        fit_ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in self.fits_d])
        h = C.c_void_p()
        rc = _lib().cpa_batch_create(n, idx, opts, lam_ptrs, fac_ptrs, fit_ptrs, int(autotune), _stream(),
                                     C.byref(h))
        _check(rc, "cpa_batch_create")
        self.h = h
        self.n = n

    def run(self):
        stats = (Stats * self.n)()
        rc = _lib().cpa_batch_run(self.h, _stream(), stats)
        _check(rc, "cpa_batch_run")
        return [s.as_dict() for s in stats]

    def fits(self):
        return [float(t.item()) for t in self.fits_d]

    def info(self):
        b = C.c_int32(0)
        cb = (C.c_int32 * 4)()
        cm = (C.c_double * 4)()
        k = C.c_int64(0)
        _check(_lib().cpa_batch_info(self.h, C.byref(b), cb, cm, C.byref(k)), "cpa_batch_info")
        return {"sm_budget": b.value, "candidates": list(cb), "candidate_ms": list(cm), "kernels": k.value}

    def free(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().cpa_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cp_arls_lev_coo(coo, factors, *, rank, samples, tau=1.0, iters=10, seed=0, fit_mode=FIT_EXACT,
                    dtype=np.float64, inplace=False, **kw) -> Result:
    """Host COO + host factors in, host results out (index built and freed inside).
    inplace=True updates the caller's factor arrays (C-contiguous float64, e.g. views
    of pinned memory) instead of copies."""
    _torch()
    s = coo_from_host(coo, dtype)
    o = default_options(rank=rank, samples=int(samples), tau=float(tau), iters=int(iters), seed=int(seed),
                        fit_mode=int(fit_mode), **kw)
    o.stream = _stream()
    if inplace:
        fs = list(factors)
        if not all(isinstance(f, np.ndarray) and f.dtype == np.float64 and f.flags.c_contiguous for f in fs):
            raise ValueError("inplace factors must be C-contiguous float64 numpy arrays")
    else:
        fs = [np.ascontiguousarray(f, dtype=np.float64).copy() for f in factors]
    lam = np.zeros(rank)
    fit = C.c_double(0.0)
    stats = Stats()
    rc = _lib().cp_arls_lev_coo(C.byref(s), C.byref(o), lam.ctypes.data,
                                _ptr_array([f.ctypes.data for f in fs]), 0, C.byref(fit), C.byref(stats))
    _check(rc, "cp_arls_lev_coo")
    return Result(lam, fs, fit.value, stats.as_dict(), rc)


def cpa_mode_update(index: Index, factors, k, *, rank, samples, tau=1.0, seed=0, it=0, precision=FP64,
                    det_cap=1 << 24, reject_cap=4096, distribution=DIST_LEVERAGE):
    """One update of mode k.  factors: CUDA float64 tensors (factor k is replaced in
    place).  Returns dict(lam, idx, cnt, wgt, sbar, sdet, attempts, pdet, warnings)."""
    torch = _torch()
    o = default_options(rank=rank, samples=int(samples), tau=float(tau), seed=int(seed),
                        precision=int(precision), det_cap=int(det_cap), reject_cap=int(reject_cap),
                        distribution=int(distribution))
    o.stream = _stream()
    s = int(samples)
    lam = torch.empty(rank, dtype=torch.float64, device="cuda")
    idx = torch.empty(s, dtype=torch.uint64, device="cuda")
    cnt = torch.empty(s, dtype=torch.int32, device="cuda")
    wgt = torch.empty(s, dtype=torch.float64, device="cuda")
    counts = (C.c_int64 * 3)()
    pdet = C.c_double(0)
    rc = _check(_lib().cpa_mode_update(index.h, C.byref(o), int(k), int(it),
                                       _ptr_array([f.data_ptr() for f in factors]), _ptr(lam), _ptr(idx),
                                       _ptr(cnt), _ptr(wgt), counts, C.byref(pdet)), "cpa_mode_update")
    sbar = counts[0]
    return dict(lam=lam, idx=idx[:sbar], cnt=cnt[:sbar], wgt=wgt[:sbar], sbar=sbar, sdet=counts[1],
                attempts=counts[2], pdet=pdet.value, warnings=rc)


# --------------------------------------------------------------------------- stages
def cpa_philox4x64(ctr, key):
    """ctr: (n, 4) uint64 CUDA tensor; key: two ints -> (n, 4) uint64 CUDA tensor."""
    torch = _torch()
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    k = (C.c_uint64 * 2)(int(key[0]), int(key[1]))
    _check(_lib().cpa_philox4x64(_ptr(ctr), k, ctr.shape[0], _ptr(out), _stream()), "cpa_philox4x64")
    return out


def cpa_leverage(A):
    torch = _torch()
    A = A.to(device="cuda", dtype=torch.float64).contiguous()
    n, r = A.shape
    lev = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = _check(_lib().cpa_leverage(_ptr(A), n, r, _ptr(lev), _stream()), "cpa_leverage")
    return lev, rc


def cpa_leverage_noalloc(A, lev=None):
    """cpa_leverage without any device allocation inside the library (the caller
    supplies the output ``lev``; the library's scratch is a fixed device array).
    A supplied ``lev`` must be a contiguous float64 tensor of n elements on A's
    device: the library writes n doubles through its pointer."""
    torch = _torch()
    A = A.to(device="cuda", dtype=torch.float64).contiguous()
    n, r = A.shape
    if lev is None:
        lev = torch.empty(n, dtype=torch.float64, device=A.device)
    else:
        if not isinstance(lev, torch.Tensor):
            raise TypeError("lev must be a torch tensor")
        if lev.dtype != torch.float64:
            raise TypeError(f"lev must be float64, not {lev.dtype}")
        if lev.device != A.device:
            raise ValueError(f"lev is on {lev.device}, A on {A.device}")
        if lev.numel() != n or not lev.is_contiguous():
            raise ValueError(f"lev must be a contiguous tensor of {n} elements")
    rc = _check(_lib().cpa_leverage_noalloc(_ptr(A), n, r, _ptr(lev), _stream()), "cpa_leverage_noalloc")
    return lev, rc


def cpa_cdf(lev, r):
    torch = _torch()
    lev = lev.to(device="cuda", dtype=torch.float64).contiguous()
    n = lev.shape[0]
    Cd = torch.empty(n, dtype=torch.uint64, device="cuda")
    info = (C.c_uint64 * 3)()
    _check(_lib().cpa_cdf(_ptr(lev), n, r, _ptr(Cd), info, _stream()), "cpa_cdf")
    return Cd, int(info[0]), int(info[1]), int(info[2])


def cpa_skrp_lev(levs, r, *, samples, tau, seed=0, it=0, mode_k=0, det_cap=1 << 24, reject_cap=4096):
    """SkrpLev over the given leverage vectors (CUDA float64 tensors, one per other
    mode).  Returns dict(idx, cnt, wgt (CUDA tensors, length sbar), sbar, sdet, attempts,
    pdet)."""
    torch = _torch()
    levs = [l.to(device="cuda", dtype=torch.float64).contiguous() for l in levs]
    d = len(levs)
    dims = np.array([l.shape[0] for l in levs], dtype=np.int64)
    s = int(samples)
    o = default_options(rank=r, samples=s, tau=float(tau), seed=int(seed), det_cap=int(det_cap),
                        reject_cap=int(reject_cap))
    o.stream = _stream()
    idx = torch.empty(s, dtype=torch.uint64, device="cuda")
    cnt = torch.empty(s, dtype=torch.int32, device="cuda")
    wgt = torch.empty(s, dtype=torch.float64, device="cuda")
    counts = (C.c_int64 * 3)()
    pdet = C.c_double(0)
    lp = _ptr_array([l.data_ptr() for l in levs])
    _check(_lib().cpa_skrp_lev(d, dims.ctypes.data, lp, r, C.byref(o), int(mode_k), int(it), _ptr(idx),
                               _ptr(cnt), _ptr(wgt), counts, C.byref(pdet)), "cpa_skrp_lev")
    sbar = counts[0]
    return dict(idx=idx[:sbar], cnt=cnt[:sbar], wgt=wgt[:sbar], sbar=sbar, sdet=counts[1],
                attempts=counts[2], pdet=pdet.value)


def cpa_sampled_mttkrp(index: Index, k, factors, idx, wgt):
    torch = _torch()
    fs = [f.to(device="cuda", dtype=torch.float64).contiguous() for f in factors]
    r = fs[0].shape[1]
    idx = idx.to(device="cuda").contiguous()
    wgt = wgt.to(device="cuda", dtype=torch.float64).contiguous()
    M = torch.empty(index.dims[k], r, dtype=torch.float64, device="cuda")
    G = torch.empty(r, r, dtype=torch.float64, device="cuda")
    nz = C.c_int64(0)
    _check(_lib().cpa_sampled_mttkrp(index.h, k, _ptr_array([f.data_ptr() for f in fs]), r, _ptr(idx),
                                     _ptr(wgt), idx.shape[0], _ptr(M), _ptr(G), C.byref(nz), _stream()),
           "cpa_sampled_mttkrp")
    return M, G, nz.value


def cpa_solve(G, M):
    torch = _torch()
    G = G.to(device="cuda", dtype=torch.float64).contiguous()
    M = M.to(device="cuda", dtype=torch.float64).contiguous()
    n, r = M.shape
    A = torch.empty_like(M)
    lam = torch.empty(r, dtype=torch.float64, device="cuda")
    rc = _check(_lib().cpa_solve(_ptr(G), _ptr(M), n, r, _ptr(A), _ptr(lam), _stream()), "cpa_solve")
    return A, lam, rc


def cpa_fit(index: Index, factors, lam):
    torch = _torch()
    fs = [f.to(device="cuda", dtype=torch.float64).contiguous() for f in factors]
    lam = lam.to(device="cuda", dtype=torch.float64).contiguous()
    out = C.c_double(0)
    _check(_lib().cpa_fit(index.h, _ptr_array([f.data_ptr() for f in fs]), _ptr(lam), lam.shape[0],
                          C.byref(out), _stream()), "cpa_fit")
    return out.value


def cpa_fit_terms(index: Index, factors, lam):
    """(||X||^2, <X, M>, ||M||^2) of Eq. 5.1 over the nonzeros of ``index``."""
    torch = _torch()
    fs = [f.to(device="cuda", dtype=torch.float64).contiguous() for f in factors]
    lam = lam.to(device="cuda", dtype=torch.float64).contiguous()
    out = (C.c_double * 3)()
    _check(_lib().cpa_fit_terms(index.h, _ptr_array([f.data_ptr() for f in fs]), _ptr(lam), lam.shape[0], out,
                                _stream()), "cpa_fit_terms")
    return float(out[0]), float(out[1]), float(out[2])


# --------------------------------------------------------------------------- estimated fit
@dataclass
class FitSample:
    """Element sample of the estimated fit (Section 5.4) on the device: coords
    (order x S int32 CUDA tensor), xs (S float64), s_nz, s_z, zero-cell attempts,
    phi = (nnz / s_nz, (prod n - nnz) / s_z)."""
    coords: object
    xs: object
    s_nz: int
    s_z: int
    attempts: int
    phi: tuple


def cpa_fit_sample(index: Index, fit_samples, alpha=0.5, seed=0, reject_cap=4096) -> FitSample:
    torch = _torch()
    coords = torch.empty((index.order, int(fit_samples)), dtype=torch.int32, device="cuda")
    xs = torch.empty(int(fit_samples), dtype=torch.float64, device="cuda")
    counts = (C.c_int64 * 3)()
    phi = (C.c_double * 2)()
    _check(_lib().cpa_fit_sample(index.h, int(fit_samples), float(alpha), int(seed), int(reject_cap),
                                 _ptr(coords), _ptr(xs), counts, phi, _stream()), "cpa_fit_sample")
    n = counts[0] + counts[1]
    return FitSample(coords[:, :n], xs[:n], counts[0], counts[1], counts[2], (phi[0], phi[1]))


def cpa_fit_estimate(index: Index, sample: FitSample, factors, lam, precision=FP64):
    """(estimated fit, F_hat) of the model [[lam; factors]] on a sample."""
    torch = _torch()
    fs = [f.to(device="cuda", dtype=torch.float64).contiguous() for f in factors]
    lam = lam.to(device="cuda", dtype=torch.float64).contiguous()
    coords = sample.coords.contiguous()
    xs = sample.xs.contiguous()
    counts = (C.c_int64 * 3)(sample.s_nz, sample.s_z, sample.attempts)
    phi = (C.c_double * 2)(*sample.phi)
    fit = C.c_double(0)
    F = C.c_double(0)
    _check(_lib().cpa_fit_estimate(index.h, _ptr(coords), _ptr(xs), counts, phi, coords.shape[1], _ptr(lam),
                                   _ptr_array([f.data_ptr() for f in fs]), lam.shape[0], int(precision),
                                   C.byref(fit), C.byref(F), _stream()), "cpa_fit_estimate")
    return fit.value, F.value


# --------------------------------------------------------------------------- range-finder init
def cpa_rrf_init(index: Index, mode, omega, seed=0):
    """Initial factor of ``mode`` (App. F): X_(k)(:, S) omega for s_init fibres drawn
    uniformly; omega: s_init x r (CUDA or CPU float64).  Returns a CUDA tensor."""
    torch = _torch()
    om = omega.to(device="cuda", dtype=torch.float64).contiguous()
    s_init, r = om.shape
    n = index.dims[mode] if 0 <= mode < index.order else 1  # an invalid mode is the library's to reject
    A = torch.empty((n, max(r, 1)), dtype=torch.float64, device="cuda")
    _check(_lib().cpa_rrf_init(index.h, int(mode), int(s_init), int(seed), _ptr(om), int(r), _ptr(A), _stream()),
           "cpa_rrf_init")
    return A
