"""Seeded synthetic inputs for CP-ARLS-LEV.

This module only makes inputs: sparse count tensors in coordinate (COO) form and
Gaussian initial factor matrices.  It holds none of the method's arithmetic and is
shared by the CUDA path's tests, the oracle's tests and the benchmark, so both sides
of every comparison see byte-identical inputs.

The real tensors of the paper (Uber, Amazon, Reddit from FROSTT, Table 6.1) are not
available; these generators stand in for them with the same shapes, nonzero counts
and the kind of value distribution the paper describes in Section 6 (counts, or
log(1 + count) for the Reddit-like tensor).  The planted-model recipe:

* component weights lambda_j ~ U[1, 2];
* factor column j of mode m is a popularity profile times a random perturbation:
  either a Dirichlet(0.1) vector (the small 60x50x40 tensor), or a Zipf(alpha)
  popularity curve (i+1)^-alpha placed under a per-component random permutation
  and multiplied by Gamma(1) noise (the large tensors);
* each event picks a component with probability proportional to lambda, then one
  index per mode from that component's columns; repeated coordinates add up to
  counts.  The number of events is raised until the nonzero count reaches the
  target (within 2 %).

All randomness comes from numpy's Philox bit generator seeded explicitly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Coo",
    "gaussian_factors",
    "planted_cp_tensor",
    "random_sparse_tensor",
    "small_planted_tensor",
    "uber_like_tensor",
    "exact_lowrank_tensor",
    "CONFIG_SMALL",
    "CONFIG_UBER",
]


@dataclass
class Coo:
    """A sparse tensor in coordinate format: ``idx[m][e]`` is the 0-based index of
    nonzero ``e`` in mode ``m`` (int32) and ``vals[e]`` its value."""

    dims: tuple
    idx: list
    vals: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def order(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])

    def as_dtype(self, dtype) -> "Coo":
        return Coo(self.dims, self.idx, self.vals.astype(dtype), dict(self.meta))

    def dense(self) -> np.ndarray:
        """Dense copy (small tensors only)."""
        X = np.zeros(self.dims, dtype=np.float64)
        X[tuple(np.asarray(i, dtype=np.int64) for i in self.idx)] = self.vals
        return X


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def gaussian_factors(dims, rank: int, seed: int = 0) -> list:
    """Initial factor matrices with standard Gaussian entries (Section 6: factor
    matrices are initialised from a standard normal distribution).  Row-major
    n_k x rank float64 arrays."""
    g = _rng(seed, 101)
    return [np.ascontiguousarray(g.standard_normal((int(n), rank))) for n in dims]


def _linear(idx_cols, dims) -> np.ndarray:
    lin = np.zeros(idx_cols[0].shape[0], dtype=np.uint64)
    stride = 1
    for col, n in zip(idx_cols, dims):
        lin += col.astype(np.uint64) * np.uint64(stride)
        stride *= int(n)
    return lin


def _unlinear(lin, dims) -> list:
    out = []
    rest = lin.copy()
    for n in dims:
        out.append((rest % np.uint64(n)).astype(np.int32))
        rest //= np.uint64(n)
    return out


def _columns(g, dims, rank, zipf_alpha, dirichlet):
    cols = []
    for n in dims:
        n = int(n)
        if zipf_alpha is None:
            C = g.dirichlet(np.full(n, dirichlet), size=rank).T  # n x rank
        else:
            base = (np.arange(n, dtype=np.float64) + 1.0) ** (-float(zipf_alpha))
            C = np.empty((n, rank))
            for j in range(rank):
                perm = g.permutation(n)
                C[:, j] = base[perm] * g.gamma(1.0, size=n)
            C /= C.sum(axis=0, keepdims=True)
        cols.append(np.ascontiguousarray(C))
    return cols


def _draw_events(g, cols, lam, events):
    rank = lam.shape[0]
    comp_counts = g.multinomial(events, lam / lam.sum())
    idx_cols = [np.empty(events, dtype=np.int64) for _ in cols]
    pos = 0
    for j in range(rank):
        c = int(comp_counts[j])
        if c == 0:
            continue
        for m, C in enumerate(cols):
            cdf = np.cumsum(C[:, j])
            cdf /= cdf[-1]
            u = g.random(c)
            idx_cols[m][pos:pos + c] = np.minimum(np.searchsorted(cdf, u, side="right"), C.shape[0] - 1)
        pos += c
    return idx_cols


def planted_cp_tensor(dims, rank, *, events=None, target_nnz=None, seed=0, zipf_alpha=None,
                      dirichlet=0.1, log_counts=False, max_rounds=12) -> Coo:
    """Count tensor drawn from a planted nonnegative CP model (see module doc).

    Give either a fixed ``events`` count, or ``target_nnz``: then the event count is
    searched (geometric then bisection on a fixed seed) until the number of distinct
    coordinates is within 2 % of the target.
    """
    dims = tuple(int(n) for n in dims)
    g0 = _rng(seed, 7)
    lam = g0.uniform(1.0, 2.0, size=rank)
    cols = _columns(g0, dims, rank, zipf_alpha, dirichlet)

    def realise(ev):
        g = _rng(seed, 11)
        idx_cols = _draw_events(g, cols, lam, int(ev))
        lin = _linear(idx_cols, dims)
        uniq, counts = np.unique(lin, return_counts=True)
        return uniq, counts

    if events is not None:
        uniq, counts = realise(events)
        ev_used = int(events)
    else:
        target = int(target_nnz)
        lo, hi = None, None
        ev = target
        uniq, counts = realise(ev)
        for _ in range(max_rounds):
            nz = uniq.shape[0]
            if abs(nz - target) <= 0.02 * target:
                break
            if nz < target:
                lo = ev
                ev = ev * 2 if hi is None else (lo + hi) // 2
            else:
                hi = ev
                ev = (lo + hi) // 2 if lo is not None else max(1, ev // 2)
            uniq, counts = realise(ev)
        ev_used = ev
    idx = _unlinear(uniq, dims)
    vals = counts.astype(np.float64)
    if log_counts:
        vals = np.log1p(vals)
    return Coo(dims, idx, vals, {"events": ev_used, "rank": rank, "seed": seed,
                                 "zipf_alpha": zipf_alpha, "lambda": lam})


def small_planted_tensor(seed: int = 0) -> Coo:
    """60 x 50 x 40 count tensor from 20,000 Poisson-process events of a planted
    rank-4 nonnegative CP model with Dirichlet(0.1) factor columns."""
    return planted_cp_tensor((60, 50, 40), 4, events=20000, seed=seed, dirichlet=0.1)


def uber_like_tensor(seed: int = 0, target_nnz: int = 3_309_490) -> Coo:
    """183 x 24 x 1140 x 1717 count tensor with about 3.31M nonzeros (the shape and
    nonzero count of the Uber tensor, Table 6.1), planted rank 25, Zipf(1.1)
    popularity."""
    return planted_cp_tensor((183, 24, 1140, 1717), 25, target_nnz=target_nnz, seed=seed,
                             zipf_alpha=1.1)


def random_sparse_tensor(dims, nnz, seed=0, dtype=np.float64, positive=True) -> Coo:
    """Uniformly random distinct coordinates with values in [0.5, 1.5) (or N(0,1))."""
    dims = tuple(int(n) for n in dims)
    g = _rng(seed, 3)
    N = math.prod(dims)
    nnz = min(int(nnz), N)
    if N <= 4 * nnz + 1024:
        lin = np.sort(g.choice(N, size=nnz, replace=False)).astype(np.uint64)
    else:
        lin = np.unique(g.integers(0, N, size=int(nnz * 1.3) + 16, dtype=np.uint64))
        lin = np.sort(g.choice(lin, size=min(nnz, lin.shape[0]), replace=False))
    idx = _unlinear(lin, dims)
    vals = g.uniform(0.5, 1.5, size=lin.shape[0]) if positive else g.standard_normal(lin.shape[0])
    return Coo(dims, idx, vals.astype(dtype), {"seed": seed})


def exact_lowrank_tensor(dims, rank, seed=0, density=0.5) -> tuple:
    """A sparse tensor that is exactly rank ``rank``: nonnegative factors with a
    fraction of zero entries, all nonzero cells of the product kept.  Returns the COO
    tensor and the planted (lambda, factors)."""
    dims = tuple(int(n) for n in dims)
    g = _rng(seed, 5)
    facs = []
    for n in dims:
        F = g.uniform(0.5, 1.5, size=(n, rank)) * (g.random((n, rank)) < density)
        # keep every row and column nonzero so the model has full rank
        for j in range(rank):
            if not F[:, j].any():
                F[g.integers(0, n), j] = 1.0
        for i in range(n):
            if not F[i].any():
                F[i, g.integers(0, rank)] = 1.0
        facs.append(F)
    lam = g.uniform(1.0, 2.0, size=rank)
    X = np.einsum("r,ir,jr,kr->ijk", lam, *facs) if len(dims) == 3 else None
    if X is None:
        # general order: build by repeated outer products
        X = np.zeros(dims)
        for j in range(rank):
            T = lam[j]
            for F in facs:
                T = np.multiply.outer(T, F[:, j])
            X += T
    nzc = np.nonzero(X)
    idx = [c.astype(np.int32) for c in nzc]
    return Coo(dims, idx, X[nzc].astype(np.float64), {"seed": seed}), lam, facs


CONFIG_SMALL = dict(name="planted-60x50x40-r4", rank=4, samples=1024, tau=1.0, iters=10, seed=0)
CONFIG_UBER = dict(name="uber-like-183x24x1140x1717-r25", rank=25, samples=2 ** 17,
                   tau=2.0 ** -17, seed=0)


def batch_specs(nprob: int = 64, seed0: int = 0, max_nnz: int = 10 ** 7) -> list:
    """The parameters of the batched workload's problems (see batch_problems): dicts
    with dims, nnz (the target count), rank, samples, tau, zipf_alpha, seed."""
    out = []
    for i in range(nprob):
        g = _rng(seed0 + i, 31)
        order = int(g.integers(3, 5))
        alpha = float(g.uniform(1.0, 1.3))
        rank = int(g.integers(5, 51))
        u = int(g.integers(14, 18))
        lg_nnz = g.uniform(4.0, np.log10(max_nnz))
        while True:
            dims = tuple(int(round(10 ** g.uniform(2.0, 5.0))) for _ in range(order))
            cells = float(np.prod([float(n) for n in dims]))
            if cells >= 2.0 ** 60:
                continue
            fewest = min(cells / n for n in dims)
            s = 2 ** u
            while s > fewest / 128 and s > 32:
                s //= 2
            if s < 16 * rank:  # far more sampled rows than unknowns per row of A_k
                continue
            # at least ~50 sampled nonzeros expected in every mode (s nnz / N_k >= 50)
            most = max(cells / n for n in dims)
            lo = max(1e4, 50.0 * most / s)
            hi = min(float(max_nnz), 0.1 * cells)
            if lo <= hi:
                break
        nnz = int(round(min(max(10 ** lg_nnz, lo), hi)))
        out.append(dict(dims=dims, nnz=nnz, rank=rank, samples=s, tau=1.0 / s, zipf_alpha=alpha, seed=seed0 + i))
    return out


def batch_problems(nprob: int = 64, seed0: int = 0, max_nnz: int = 10 ** 6) -> list:
    """The batched workload: independent 3- and 4-way planted count tensors of uneven
    size.  Problem i (seed seed0 + i): order 3 or 4; mode sizes log-uniform in
    [10^2, 10^5] (redrawn while their product reaches 2^60, or while no nonzero count
    fits the bounds below); nnz log-uniform in [10^4, max_nnz], at most a tenth of the
    cells and at least 50 N_k / s for every mode k (N_k = Khatri-Rao rows), so that
    the sampled right-hand sides are not empty; Zipf(alpha) popularity with alpha
    uniform in [1.0, 1.3]; CP rank uniform in 5..50; s = 2^u, u uniform in 14..17,
    lowered to a power of two at most 1/128 of the fewest Khatri-Rao rows of any mode
    (the method's regime s << N_k: with s near N_k and skewed leverage almost all of the
    mass is deterministic and the rejection loop of Alg. 2 rarely finds a row below
    tau) and at least 16 r (mode sizes redrawn otherwise); tau = 1/s.  Returns dicts with coo, rank, samples, tau, zipf_alpha, seed."""
    out = []
    for sp in batch_specs(nprob, seed0, max_nnz):
        coo = planted_cp_tensor(sp["dims"], sp["rank"], target_nnz=sp["nnz"], seed=sp["seed"],
                                zipf_alpha=sp["zipf_alpha"])
        out.append(dict(coo=coo, rank=sp["rank"], samples=sp["samples"], tau=sp["tau"], zipf_alpha=sp["zipf_alpha"],
                        seed=sp["seed"]))
    return out
