"""The host side of the sharded run on the CPU: slice ranges partition the nonzeros
with balanced counts, and the exchange (the sum of the ranks' partial M) gives every
one of two gloo ranks the same sum, equal to the sum computed in one process."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import synth  # noqa: E402
from paper_2006_16438_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slice_bounds_partition_and_balance():
    coo = synth.planted_cp_tensor((500, 40, 30), 5, target_nnz=20000, seed=2, zipf_alpha=1.2)
    for nr in (1, 2, 3, 7):
        b = shard.slice_bounds(coo.idx[0], 500, nr)
        assert b[0] == 0 and b[-1] == 500 and all(x <= y for x, y in zip(b, b[1:]))
        parts = [shard.shard_coo(coo, b, q) for q in range(nr)]
        assert sum(p.nnz for p in parts) == coo.nnz
        for q, p in enumerate(parts):
            assert np.all((p.idx[0] >= b[q]) & (p.idx[0] < b[q + 1]))
            assert p.dims == coo.dims
        keys = np.sort(np.concatenate([np.ravel_multi_index(p.idx, coo.dims) for p in parts]))
        np.testing.assert_array_equal(keys, np.sort(np.ravel_multi_index(coo.idx, coo.dims)))
        # no slice range is more than one heaviest slice above the mean
        heaviest = np.bincount(coo.idx[0], minlength=500).max()
        assert max(p.nnz for p in parts) <= coo.nnz / nr + heaviest


def _partial(rank):
    g = np.random.default_rng(100 + rank)
    return torch.from_numpy(g.standard_normal((37, 6)))


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M = _partial(rank)
        terms = torch.tensor([1.5 + rank, 0.25 * rank], dtype=torch.float64)
        shard.allreduce_sum([M, terms])
        out[rank] = (M.numpy().copy(), terms.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_partial_m():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    expect = (_partial(0) + _partial(1)).numpy()
    for rank in range(world):
        np.testing.assert_allclose(res[rank][0], expect, rtol=0, atol=1e-15)
        np.testing.assert_allclose(res[rank][1], [4.0, 0.25], rtol=0, atol=0)
    np.testing.assert_array_equal(res[0][0], res[1][0])


def test_local_sum_in_shard_order():
    parts = [[torch.full((3,), float(q + 1))] for q in range(3)]
    shard.local_sum(parts)
    for p in parts:
        np.testing.assert_array_equal(p[0].numpy(), [6.0, 6.0, 6.0])
