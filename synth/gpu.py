"""Seeded planted-CP count tensors generated on the GPU (torch), for sizes the CPU
generator cannot reach (billions of nonzeros).

Model (as ``synth.planted_cp_tensor`` with Zipf columns): component weights
lam_j ~ U[1, 2]; column j of mode m is Zipf(alpha) popularity under a seeded
permutation times Gamma(1) noise, normalised; an event picks component j with
probability lam_j / sum(lam) and then index i_m from column j of every mode; the value
at a coordinate is its number of events (optionally log(1 + count)).

The tensor is generated slice by slice over ranges of mode-0 indices: each range gets
its multinomial share of the events (its probability mass), the events of a range are
drawn with mode-0 indices restricted to it, and duplicates are merged inside the
range.  Ranges are disjoint in i_0, so the coordinates are globally unique without a
global sort, and the in-range linear key fits 63 bits.  Output: int32 index tensors
and float32 values on the device, in ascending (i_0, i_1, ..., i_{d-1}) order.

This module holds none of the decomposition's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np


def _columns_gpu(torch, gen, n, rank, alpha, device):
    """n x rank column weights (float64, columns sum to 1)."""
    base = (torch.arange(n, device=device, dtype=torch.float64) + 1.0) ** (-float(alpha))
    C = torch.empty((n, rank), device=device, dtype=torch.float64)
    for j in range(rank):
        perm = torch.randperm(n, device=device, generator=gen)
        u = torch.rand(n, device=device, dtype=torch.float64, generator=gen)
        C[:, j] = base[perm] * (-torch.log1p(-u))  # Gamma(1) = Exp(1)
    C /= C.sum(dim=0, keepdim=True)
    return C


def _flat_cdf(torch, W, device):
    """Per-column cumulative sums of W (rows x rank) placed at offsets j (column j's
    CDF occupies [j, j + 1]), as one ascending vector."""
    rows, rank = W.shape
    cdf = torch.cumsum(W, dim=0)
    cdf = cdf / cdf[-1:, :].clamp_min(1e-300)
    return (cdf + torch.arange(rank, device=device, dtype=torch.float64)[None, :]).t().contiguous().view(-1)


def _draw_by_component(torch, gen, W, comp, device, flat=None):
    """Index per event from column comp[e] of the weight matrix W (rows x rank):
    inverse CDF on the flat per-column CDF (computed here unless given), one search
    for all events."""
    rows, rank = W.shape
    if flat is None:
        flat = _flat_cdf(torch, W, device)
    u = torch.rand(comp.shape[0], device=device, dtype=torch.float64, generator=gen)
    pos = torch.searchsorted(flat, comp.to(torch.float64) + u, right=True)
    idx = pos - comp * rows
    return idx.clamp_(0, rows - 1)


def planted_cp_tensor_gpu(dims, rank, *, events, seed=0, zipf_alpha=1.1, log_counts=False,
                          events_per_slice=1 << 26, device="cuda"):
    """Returns (idx, vals): a list of int32 device tensors (one per mode) and a float32
    device tensor of values.  ``events`` Poisson events are drawn in total."""
    import torch
    dims = [int(n) for n in dims]
    d = len(dims)
    g_host = np.random.Generator(np.random.Philox(key=[seed, 211]))
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 17)
    lam = torch.tensor(g_host.uniform(1.0, 2.0, size=rank), device=device, dtype=torch.float64)
    cols = [_columns_gpu(torch, gen, n, rank, zipf_alpha, device) for n in dims]
    # mode-0 ranges: at most events_per_slice events each, and an in-range key below 2^63
    others = 1
    for n in dims[1:]:
        others *= n
    max_width = max(1, (2 ** 63 - 1) // others)
    n0 = dims[0]
    nslices = max(math.ceil(events / events_per_slice), math.ceil(n0 / max_width), 1)
    bounds = np.linspace(0, n0, nslices + 1).round().astype(np.int64)
    C0 = cols[0]
    w = lam / lam.sum()
    # probability mass of every range, per component: sum_{i0 in range} C0(i0, j) w_j
    csum = torch.cumsum(C0, dim=0)
    starts = torch.tensor(bounds[:-1], device=device)
    ends = torch.tensor(bounds[1:], device=device)
    hi = csum[ends - 1]
    lo = torch.where(starts[:, None] > 0, csum[(starts - 1).clamp_min(0)], torch.zeros_like(hi))
    mass = (hi - lo) * w[None, :]  # nslices x rank
    per_slice = g_host.multinomial(int(events), (mass.sum(dim=1) / mass.sum()).cpu().numpy())
    flats = [None] + [_flat_cdf(torch, cols[m], device) for m in range(1, d)]  # same for every slice
    out_idx = [[] for _ in range(d)]
    out_val = []
    for sl in range(nslices):
        e = int(per_slice[sl])
        a, b = int(bounds[sl]), int(bounds[sl + 1])
        if e == 0 or b <= a:
            continue
        pj = (mass[sl] / mass[sl].sum()).cpu().numpy()
        counts = g_host.multinomial(e, pj / pj.sum())
        comp = torch.repeat_interleave(torch.arange(rank, device=device),
                                       torch.tensor(counts, device=device))
        i0 = _draw_by_component(torch, gen, C0[a:b], comp, device) + a
        key = i0 - a
        rest = []
        for m in range(1, d):
            im = _draw_by_component(torch, gen, cols[m], comp, device, flats[m])
            key = key * dims[m] + im
            rest.append(im)
        uniq, cnt = torch.unique(key, sorted=True, return_counts=True)
        # decode the in-range key (mode d-1 fastest)
        coords = []
        r = uniq
        for m in range(d - 1, 0, -1):
            coords.append((r % dims[m]).to(torch.int32))
            r = r // dims[m]
        coords.append((r + a).to(torch.int32))
        coords.reverse()
        for m in range(d):
            out_idx[m].append(coords[m])
        v = cnt.to(torch.float32)
        out_val.append(torch.log1p(v) if log_counts else v)
        del comp, i0, key, rest, uniq, cnt
    del flats
    idx = []
    for m in range(d):  # one mode at a time, dropping its slices: peak about 1 + 1/(d + 1) tensors
        idx.append(torch.cat(out_idx[m]))
        out_idx[m] = None
    vals = torch.cat(out_val)
    del out_val
    return idx, vals


def batch_problems_gpu(nprob=64, seed0=0, max_nnz=10 ** 7, device="cuda"):
    """The batched workload of ``synth.batch_specs`` generated on the GPU: per problem
    the planted model's tensor from 1.3 events per target nonzero (duplicates merged,
    so the count lands near the target), as (spec, idx, vals) with device tensors."""
    import synth
    out = []
    for sp in synth.batch_specs(nprob, seed0, max_nnz):
        idx, vals = planted_cp_tensor_gpu(sp["dims"], sp["rank"], events=int(1.3 * sp["nnz"]), seed=sp["seed"],
                                          zipf_alpha=sp["zipf_alpha"], device=device)
        out.append((sp, idx, vals))
    return out
