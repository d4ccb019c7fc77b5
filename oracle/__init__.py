"""Python access to the plain FP64 CPU oracle (``oracle/cpa_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use this package.  The CUDA library never
imports, links or calls it, and it never calls the CUDA library.

The C source is compiled on first use with gcc (``-O2 -ffp-contract=off`` so that no
multiply-add is fused and the sampling arithmetic is the IEEE sequence the source
states) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpa_oracle.c")
_HDR = os.path.join(_HERE, "cpa_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_handle = None

OK = 0
ERR_ARG = -1
ERR_COO_RANGE = -2
ERR_COO_DUP = -3
ERR_OOM = -4
ERR_REJECT_LIMIT = -5
ERR_DET_CAP = -6
DIST_LEVERAGE = 0
DIST_UNIFORM = 1
DIST_LENGTH_SQUARED = 2
WARN_SINGULAR_GRAM = 1
WARN_RANK_DEFICIENT_LEV = 2


class OracleError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"oracle error {code} {what}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def _lib():
    global _handle
    if _handle is None:
        path = build()
        lib = C.CDLL(path)
        _declare(lib)
        _handle = lib
    return _handle


P = C.c_void_p
I64 = C.c_int64
U64 = C.c_uint64
I32 = C.c_int


def _declare(lib):
    lib.orc_philox4x64_10.argtypes = [P, P, P]
    lib.orc_philox4x64_10.restype = None
    lib.orc_leverage.argtypes = [P, I64, I32, P, P]
    lib.orc_leverage.restype = I32
    lib.orc_cdf.argtypes = [P, I64, I32, P, P, P, P]
    lib.orc_cdf.restype = U64
    lib.orc_draw.argtypes = [P, I64, U64, U64]
    lib.orc_draw.restype = I64
    lib.orc_exact_sum.argtypes = [P, I64]
    lib.orc_exact_sum.restype = C.c_double
    lib.orc_det_skrp.argtypes = [P, C.c_double, I64, I64, P, P, P, P]
    lib.orc_det_skrp.restype = I32
    lib.orc_rnd_skrp.argtypes = [P, I64, C.c_double, C.c_double, U64, U64, I32, I32, P, P, P]
    lib.orc_rnd_skrp.restype = I32
    lib.orc_skrp_lev.argtypes = [P, I64, C.c_double, U64, U64, I32, I64, I32, P, P, P, P, P, P, P]
    lib.orc_skrp_lev.restype = I32
    lib.orc_index_build.argtypes = [I32, P, I64, P, P, P]
    lib.orc_index_build.restype = I32
    lib.orc_index_free.argtypes = [P]
    lib.orc_index_free.restype = None
    lib.orc_index_nfib.argtypes = [P, I32]
    lib.orc_index_nfib.restype = I64
    lib.orc_index_export.argtypes = [P, I32, P, P, P, P]
    lib.orc_index_export.restype = None
    lib.orc_sampled_mttkrp.argtypes = [P, I32, P, I32, P, P, I64, P, P, P]
    lib.orc_sampled_mttkrp.restype = I32
    lib.orc_exact_mttkrp.argtypes = [P, I32, P, I32, P, P]
    lib.orc_exact_mttkrp.restype = I32
    lib.orc_solve.argtypes = [P, P, I64, I32, P]
    lib.orc_solve.restype = I32
    lib.orc_normalize.argtypes = [P, I64, I32, P]
    lib.orc_normalize.restype = None
    lib.orc_fit.argtypes = [P, P, P, I32]
    lib.orc_fit.restype = C.c_double
    lib.orc_cp_arls_lev.argtypes = [P, I32, I64, C.c_double, I32, I32, I32, C.c_double, U64, U64,
                                    I64, I32, P, P, P, P, I32]
    lib.orc_cp_arls_lev.restype = I32
    lib.orc_mode_update_once.argtypes = [P, I32, I32, P, P, I64, C.c_double, U64, U64, I64, I32,
                                         P, P, P, P, P, I32]
    lib.orc_mode_update_once.restype = I32
    lib.orc_cp_als.argtypes = [P, I32, I32, P, P, P]
    lib.orc_cp_als.restype = I32
    lib.orc_rrf_init.argtypes = [P, I32, I64, U64, P, I32, P]
    lib.orc_rrf_init.restype = I32
    lib.orc_scores.argtypes = [P, I64, I32, I32, P, P]
    lib.orc_scores.restype = I32
    lib.orc_fit_sample.argtypes = [P, I64, C.c_double, U64, I32, P, P, P, P]
    lib.orc_fit_sample.restype = I32
    lib.orc_fit_estimate.argtypes = [P, P, P, P, P, I64, P, P, I32, P]
    lib.orc_fit_estimate.restype = C.c_double


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr_array(arrs):
    arr = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return arr


# --------------------------------------------------------------------------- basics
def philox4x64_10(ctr, key):
    """Philox4x64-10 block: ctr (4,) uint64, key (2,) uint64 -> (4,) uint64."""
    c = _c(ctr, np.uint64)
    k = _c(key, np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def leverage(A):
    """Leverage scores of the rows of A by pivoted Householder QR; returns (lev, rank)."""
    A = _c(A, np.float64)
    n, r = A.shape
    lev = np.zeros(n)
    rank = C.c_int(0)
    rc = _lib().orc_leverage(_ptr(A), n, r, _ptr(lev), C.byref(rank))
    if rc < 0:
        raise OracleError(rc, "leverage")
    return lev, rank.value


class ModeDist:
    """Fixed-point sampling distribution of one mode (q, inclusive CDF C, T, ...)."""

    def __init__(self, lev, r):
        lev = _c(lev, np.float64)
        n = lev.shape[0]
        self.n = n
        self.q = np.zeros(n, dtype=np.uint64)
        self.C = np.zeros(n, dtype=np.uint64)
        mx = C.c_uint64(0)
        nz = C.c_int64(0)
        self.T = int(_lib().orc_cdf(_ptr(lev), n, r, _ptr(self.q), _ptr(self.C), C.byref(mx),
                                    C.byref(nz)))
        self.maxq = int(mx.value)
        self.nnzq = int(nz.value)

    @property
    def p(self):
        """p_m(i) = q_i / T as float64 (the probabilities the sampler uses)."""
        return self.q.astype(np.float64) / float(self.T)


def draw(dist: ModeDist, u: int) -> int:
    return int(_lib().orc_draw(_ptr(dist.C), dist.n, dist.T, int(u)))


def exact_sum(x):
    x = _c(x, np.float64)
    return float(_lib().orc_exact_sum(_ptr(x), x.shape[0]))


class _Sampler(C.Structure):
    _fields_ = [("d", C.c_int), ("n", P), ("C", P), ("T", P), ("maxq", P), ("nnzq", P)]


def _sampler(dists):
    n = np.array([d.n for d in dists], dtype=np.int64)
    T = np.array([d.T for d in dists], dtype=np.uint64)
    mq = np.array([d.maxq for d in dists], dtype=np.uint64)
    nz = np.array([d.nnzq for d in dists], dtype=np.int64)
    Cp = _ptr_array([d.C for d in dists])
    S = _Sampler(len(dists), n.ctypes.data, C.cast(Cp, C.c_void_p), T.ctypes.data,
                 mq.ctypes.data, nz.ctypes.data)
    S._keep = (n, T, mq, nz, Cp, dists)
    return S


def det_skrp(dists, tau, s, cap=1 << 24):
    """DetSkrp: (idet keys ascending, p values, s_det, p_det)."""
    S = _sampler(dists)
    idet = np.zeros(max(1, min(cap, 1 << 26)), dtype=np.uint64)
    pv = np.zeros_like(idet, dtype=np.float64)
    sdet = C.c_int64(0)
    pdet = C.c_double(0)
    rc = _lib().orc_det_skrp(C.byref(S), float(tau), int(s), int(cap), _ptr(idet), _ptr(pv),
                             C.byref(sdet), C.byref(pdet))
    if rc < 0:
        raise OracleError(rc, "det_skrp")
    k = sdet.value
    return idet[:k].copy(), pv[:k].copy(), k, pdet.value


def rnd_skrp(dists, srnd, tau, pdet, seed, it, mode_k, reject_cap=4096):
    """RndSkrp: (irnd per slot, wrnd per slot, attempts)."""
    S = _sampler(dists)
    irnd = np.zeros(max(1, srnd), dtype=np.uint64)
    wrnd = np.zeros(max(1, srnd))
    att = C.c_int64(0)
    rc = _lib().orc_rnd_skrp(C.byref(S), int(srnd), float(tau), float(pdet), int(seed), int(it),
                             int(mode_k), int(reject_cap), _ptr(irnd), _ptr(wrnd), C.byref(att))
    if rc < 0:
        raise OracleError(rc, "rnd_skrp")
    return irnd[:srnd].copy(), wrnd[:srnd].copy(), att.value


def skrp_lev(dists, s, tau, seed, it, mode_k, det_cap=1 << 24, reject_cap=4096):
    """SkrpLev (Alg. 1): dict with idx, cnt, wgt, sbar, sdet, pdet, attempts."""
    S = _sampler(dists)
    idx = np.zeros(s, dtype=np.uint64)
    cnt = np.zeros(s, dtype=np.uint32)
    wgt = np.zeros(s)
    sbar = C.c_int64(0)
    sdet = C.c_int64(0)
    pdet = C.c_double(0)
    att = C.c_int64(0)
    rc = _lib().orc_skrp_lev(C.byref(S), int(s), float(tau), int(seed), int(it), int(mode_k),
                             int(det_cap), int(reject_cap), _ptr(idx), _ptr(cnt), _ptr(wgt),
                             C.byref(sbar), C.byref(sdet), C.byref(pdet), C.byref(att))
    if rc < 0:
        raise OracleError(rc, "skrp_lev")
    k = sbar.value
    return dict(idx=idx[:k].copy(), cnt=cnt[:k].copy(), wgt=wgt[:k].copy(), sbar=k,
                sdet=sdet.value, pdet=pdet.value, attempts=att.value)


# --------------------------------------------------------------------------- tensor
class Index:
    """Per-mode fibre index of a COO tensor (owned by the oracle library)."""

    def __init__(self, coo):
        self.dims = tuple(int(n) for n in coo.dims)
        self.order = len(self.dims)
        self._idx = [_c(i, np.int32) for i in coo.idx]
        self._val = _c(coo.vals, np.float64)
        self.nnz = self._val.shape[0]
        d = np.array(self.dims, dtype=np.int64)
        self._dims = d
        ip = _ptr_array(self._idx)
        self._ip = ip
        h = C.c_void_p(0)
        rc = _lib().orc_index_build(self.order, _ptr(d), self.nnz, C.cast(ip, C.c_void_p),
                                    _ptr(self._val), C.byref(h))
        if rc < 0:
            raise OracleError(rc, "index_build")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            _lib().orc_index_free(h)
            self.h = None

    def nfib(self, k):
        return int(_lib().orc_index_nfib(self.h, k))

    def export(self, k):
        F = self.nfib(k)
        keys = np.zeros(F, dtype=np.uint64)
        off = np.zeros(F + 1, dtype=np.int64)
        ik = np.zeros(self.nnz, dtype=np.int32)
        val = np.zeros(self.nnz)
        _lib().orc_index_export(self.h, k, _ptr(keys), _ptr(off), _ptr(ik), _ptr(val))
        return keys, off, ik, val


def _factor_ptrs(factors):
    fs = [_c(A, np.float64) for A in factors]
    return fs, _ptr_array(fs)


def sampled_mttkrp(index: Index, k, factors, idx, wgt):
    fs, fp = _factor_ptrs(factors)
    r = fs[0].shape[1]
    idx = _c(idx, np.uint64)
    wgt = _c(wgt, np.float64)
    M = np.zeros((index.dims[k], r))
    G = np.zeros((r, r))
    nz = C.c_int64(0)
    _lib().orc_sampled_mttkrp(index.h, k, C.cast(fp, C.c_void_p), r, _ptr(idx), _ptr(wgt),
                              idx.shape[0], _ptr(M), _ptr(G), C.byref(nz))
    return M, G, nz.value


def exact_mttkrp(index: Index, k, factors):
    fs, fp = _factor_ptrs(factors)
    r = fs[0].shape[1]
    M = np.zeros((index.dims[k], r))
    G = np.zeros((r, r))
    _lib().orc_exact_mttkrp(index.h, k, C.cast(fp, C.c_void_p), r, _ptr(M), _ptr(G))
    return M, G


def solve(G, M):
    G = _c(G, np.float64)
    M = _c(M, np.float64)
    n, r = M.shape
    A = np.zeros((n, r))
    rc = _lib().orc_solve(_ptr(G), _ptr(M), n, r, _ptr(A))
    return A, rc


def normalize(A):
    A = _c(A, np.float64).copy()
    n, r = A.shape
    lam = np.zeros(r)
    _lib().orc_normalize(_ptr(A), n, r, _ptr(lam))
    return A, lam


def fit(index: Index, factors, lam):
    fs, fp = _factor_ptrs(factors)
    lam = _c(lam, np.float64)
    return float(_lib().orc_fit(index.h, C.cast(fp, C.c_void_p), _ptr(lam), lam.shape[0]))


class FitSample:
    """Stratified element sample of the estimated fit (Section 5.4): coords
    (order x S int32), xs (S values, nonzero samples first), s_nz, s_z, zero attempts
    and the weights phi = (nnz / s_nz, (prod n - nnz) / s_z)."""

    def __init__(self, coords, xs, counts, phi):
        self.coords, self.xs = coords, xs
        self.s_nz, self.s_z, self.attempts = (int(c) for c in counts)
        self.phi = phi


def fit_sample(index: Index, s_fit, alpha=0.5, seed=0, reject_cap=4096) -> FitSample:
    coords = np.zeros((index.order, int(s_fit)), dtype=np.int32)
    xs = np.zeros(int(s_fit))
    counts = np.zeros(3, dtype=np.int64)
    phi = np.zeros(2)
    rc = _lib().orc_fit_sample(index.h, int(s_fit), float(alpha), int(seed), int(reject_cap), _ptr(coords),
                               _ptr(xs), _ptr(counts), _ptr(phi))
    if rc < 0:
        raise OracleError(rc, "fit_sample")
    S = int(counts[0] + counts[1])
    return FitSample(coords[:, :S].copy(), xs[:S].copy(), counts, phi)


def fit_estimate(index: Index, sample: FitSample, factors, lam):
    """(estimated fit 1 - sqrt(F_hat) / ||X||, F_hat) of Section 5.4."""
    fs, fp = _factor_ptrs(factors)
    lam = _c(lam, np.float64)
    coords = _c(sample.coords, np.int32)
    xs = _c(sample.xs, np.float64)
    counts = np.array([sample.s_nz, sample.s_z, sample.attempts], dtype=np.int64)
    phi = _c(sample.phi, np.float64)
    F = C.c_double(0.0)
    f = _lib().orc_fit_estimate(index.h, _ptr(coords), _ptr(xs), _ptr(counts), _ptr(phi), coords.shape[1],
                                C.cast(fp, C.c_void_p), _ptr(lam), lam.shape[0], C.byref(F))
    return float(f), F.value


def rrf_init(index: Index, k, omega, seed=0):
    """Randomized range finder initial factor of mode k (App. F): X_(k)(:, S) omega."""
    omega = _c(omega, np.float64)
    s_init, r = omega.shape
    A = np.zeros((index.dims[k], r))
    rc = _lib().orc_rrf_init(index.h, int(k), int(s_init), int(seed), _ptr(omega), int(r), _ptr(A))
    if rc < 0:
        raise OracleError(rc, "rrf_init")
    return A


def scores(A, dist=DIST_LEVERAGE):
    """Row scores (summing to the rank) of the chosen per-factor distribution."""
    A = _c(A, np.float64)
    n, r = A.shape
    out = np.zeros(n)
    rank = C.c_int(0)
    rc = _lib().orc_scores(_ptr(A), n, r, int(dist), _ptr(out), C.byref(rank))
    if rc < 0:
        raise OracleError(rc, "scores")
    return out, rank.value


def cp_arls_lev(index: Index, factors, *, rank, samples, tau=1.0, iters=10, epoch_len=5,
                patience=3, tol=0.0, seed=0, iter_offset=0, det_cap=1 << 24, reject_cap=4096,
                distribution=DIST_LEVERAGE):
    """Alg. 3.  Returns (lambda, factors, fit, iters_done, warnings)."""
    fs = [_c(A, np.float64).copy() for A in factors]
    fp = _ptr_array(fs)
    lam = np.zeros(rank)
    f = C.c_double(0)
    done = C.c_int(0)
    rc = _lib().orc_cp_arls_lev(index.h, rank, int(samples), float(tau), int(iters), int(epoch_len),
                                int(patience), float(tol), int(seed), int(iter_offset),
                                int(det_cap), int(reject_cap), C.cast(fp, C.c_void_p), _ptr(lam),
                                C.byref(f), C.byref(done), int(distribution))
    if rc < 0:
        raise OracleError(rc, "cp_arls_lev")
    return lam, fs, f.value, done.value, rc


def mode_update(index: Index, factors, k, *, rank, samples, tau=1.0, seed=0, it=0,
                det_cap=1 << 24, reject_cap=4096, distribution=DIST_LEVERAGE):
    """One randomized update of mode k from the given factors (Alg. 3 inner loop).
    Returns dict(A=new factor k (normalised), lam, idx, cnt, wgt, sbar, sdet, pdet,
    nnz_sampled, attempts, warnings)."""
    fs = [_c(A, np.float64).copy() for A in factors]
    fp = _ptr_array(fs)
    lam = np.zeros(rank)
    s = int(samples)
    idx = np.zeros(s, dtype=np.uint64)
    cnt = np.zeros(s, dtype=np.uint32)
    wgt = np.zeros(s)
    st = np.zeros(4, dtype=np.int64)
    pdet = C.c_double(0)
    rc = _lib().orc_mode_update_once(index.h, rank, int(k), C.cast(fp, C.c_void_p), _ptr(lam), s,
                                     float(tau), int(seed), int(it), int(det_cap), int(reject_cap),
                                     _ptr(idx), _ptr(cnt), _ptr(wgt), _ptr(st), C.byref(pdet),
                                     int(distribution))
    if rc < 0:
        raise OracleError(rc, "mode_update")
    sbar = int(st[0])
    return dict(A=fs[k], lam=lam, idx=idx[:sbar].copy(), cnt=cnt[:sbar].copy(),
                wgt=wgt[:sbar].copy(), sbar=sbar, sdet=int(st[1]), pdet=pdet.value,
                nnz_sampled=int(st[2]), attempts=int(st[3]), warnings=rc)


def cp_als(index: Index, factors, *, rank, iters=10):
    fs = [_c(A, np.float64).copy() for A in factors]
    fp = _ptr_array(fs)
    lam = np.zeros(rank)
    f = C.c_double(0)
    rc = _lib().orc_cp_als(index.h, rank, int(iters), C.cast(fp, C.c_void_p), _ptr(lam),
                           C.byref(f))
    return lam, fs, f.value, rc


def mode_dists(factors, r, skip=None):
    """Leverage-derived sampling distributions of every mode except ``skip``."""
    out = []
    for m, A in enumerate(factors):
        if m == skip:
            continue
        lev, _ = leverage(A)
        out.append(ModeDist(lev, r))
    return out
