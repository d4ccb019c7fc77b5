"""Alg. 3 with the tensor's nonzeros split over ranks (one process per GPU).

The sampled least-squares step shards without changing what it computes (the
paper's closing discussion of a distributed variant keeps the factor matrices in
one place and gathers the sampled fibres):

* the factor matrices are replicated on every rank;
* every rank draws the same sampled Khatri-Rao rows: the draws depend only on the
  replicated factors' leverage distributions and on counter-based Philox counters
  (seed, iteration, mode, slot, attempt), so no samples are exchanged;
* rank q holds the nonzeros whose mode-0 index lies in its slice range
  [bounds[q], bounds[q + 1]) and builds the fibre index of those alone, so its
  sampled MTTKRP covers exactly its part of X~_(k) (every sampled fibre splits into
  the ranks' pieces);
* one exchange per mode update: the sum of the ranks' partial M over the ranks
  (an all-reduce); the sampled Gram depends on the samples only and is the same on
  every rank, so every rank solves the same normal equations and keeps the same
  factors, bit for bit;
* the fit (Eq. 5.1) adds the ranks' ||X_q||^2 and <X_q, M> (a second all-reduce,
  once per fit).

The orchestration here is host logic; every step of the arithmetic runs in the CUDA
library through its stage entry points (cpa_leverage, cpa_skrp_lev,
cpa_sampled_mttkrp, cpa_solve, cpa_fit_terms).  The exchange is a callable that sums
a list of per-rank tensors in place: ``allreduce_sum`` (torch.distributed, NCCL on
GPUs or gloo on CPU tensors) across processes, or ``local_sum`` when one process
holds several shards (the single-GPU tests).
"""
from __future__ import annotations

import math

import numpy as np


def slice_bounds(mode0_index, n0, nranks):
    """Mode-0 index bounds (nranks + 1 ascending values, 0 .. n0) that split the
    nonzeros into nranks slice ranges of near-equal nonzero counts."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    counts = np.bincount(np.asarray(mode0_index, dtype=np.int64), minlength=int(n0))
    cum = np.concatenate([[0], np.cumsum(counts)])
    total = int(cum[-1])
    bounds = [0]
    for q in range(1, nranks):
        target = total * q / nranks
        b = int(np.searchsorted(cum, target, side="left"))
        bounds.append(min(max(b, bounds[-1]), int(n0)))
    bounds.append(int(n0))
    return bounds


def shard_coo(coo, bounds, rank):
    """The nonzeros of rank ``rank``'s slice range, same dimensions (a synth.Coo-like
    object with dims, idx, vals)."""
    lo, hi = bounds[rank], bounds[rank + 1]
    i0 = np.asarray(coo.idx[0])
    sel = (i0 >= lo) & (i0 < hi)
    return type(coo)(coo.dims, [np.ascontiguousarray(np.asarray(c)[sel]) for c in coo.idx],
                     np.ascontiguousarray(np.asarray(coo.vals)[sel]))


def allreduce_sum(tensors, group=None):
    """Sum each tensor over the ranks of the process group, in place (one all-reduce
    per tensor: NCCL for CUDA tensors, gloo for CPU tensors)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def local_sum(parts):
    """The exchange when one process holds all shards: parts[q] is shard q's list of
    tensors; every shard's tensors are replaced by the sum over shards, added in
    shard order."""
    for i in range(len(parts[0])):
        acc = parts[0][i].clone()
        for q in range(1, len(parts)):
            acc += parts[q][i]
        for q in range(len(parts)):
            parts[q][i].copy_(acc)
    return parts


class ShardedRun:
    """CP-ARLS-LEV (Alg. 3, fixed number of outer iterations, FP64) over the shards
    this process holds.

    indices: the fibre indices of this process's shards (one per shard; one on a real
    rank, several when one process emulates the ranks); factors: replicated initial
    factor matrices (CUDA float64 tensors, n_m x r); exchange: a callable taking a
    list (per shard) of lists of tensors and summing them over all shards of all
    ranks in place (``local_sum``, or ``lambda parts: [allreduce_sum(p) for p in
    parts]`` with one shard per rank)."""

    def __init__(self, indices, factors, *, rank, samples, tau, seed=0, exchange=None):
        import torch
        from . import binding
        self.b = binding
        self.indices = list(indices)
        self.r = int(rank)
        self.s = int(samples)
        self.tau = float(tau)
        self.seed = int(seed)
        self.exchange = exchange or local_sum
        self.factors = [f.detach().to(device="cuda", dtype=torch.float64).contiguous().clone() for f in factors]
        self.dims = [int(f.shape[0]) for f in self.factors]
        self.lam = torch.ones(self.r, dtype=torch.float64, device="cuda")
        self.levs = [binding.cpa_leverage(f)[0] for f in self.factors]
        self.it = 0
        self.last = {}

    def update(self, k, it):
        """One update of mode k at global outer iteration it: the same samples on every
        shard, the partial M of each shard, their sum, the shared solve."""
        b = self.b
        levs = [self.levs[m] for m in range(len(self.dims)) if m != k]
        smp = b.cpa_skrp_lev(levs, self.r, samples=self.s, tau=self.tau, seed=self.seed, it=it, mode_k=k)
        parts, G = [], None
        nz = 0
        for ix in self.indices:
            M, Gq, nzq = b.cpa_sampled_mttkrp(ix, k, self.factors, smp["idx"], smp["wgt"])
            parts.append([M])
            G = Gq if G is None else G
            nz += nzq
        self.exchange(parts)
        A, lam, warn = b.cpa_solve(G, parts[0][0])
        self.factors[k] = A
        self.lam = lam
        self.levs[k] = b.cpa_leverage(A)[0]
        self.last = dict(sbar=smp["sbar"], sdet=smp["sdet"], idx=smp["idx"], nnz_sampled_local=nz, M=parts[0][0],
                         G=G, warnings=warn)
        return self.last

    def iterate(self, iters):
        for _ in range(int(iters)):
            for k in range(len(self.dims)):
                self.update(k, self.it)
            self.it += 1
        return self

    def fit(self):
        """Eq. 5.1 from the shards' summed ||X_q||^2 and <X_q, M> and the shared ||M||^2."""
        import torch
        b = self.b
        parts = []
        m2 = 0.0
        for ix in self.indices:
            x2, inner, m2 = b.cpa_fit_terms(ix, self.factors, self.lam)
            parts.append([torch.tensor([x2, inner], dtype=torch.float64, device="cuda")])
        self.exchange(parts)
        x2, inner = (float(v) for v in parts[0][0].cpu())
        f2 = max(0.0, x2 - 2.0 * inner + m2)
        return 1.0 - math.sqrt(f2) / math.sqrt(x2) if x2 > 0 else 0.0
