"""The sharded run on one GPU: the tensor's nonzeros split into mode-0 slice ranges,
one fibre index per shard, the same samples on every shard, the shards' partial M
summed (the exchange of a multi-GPU run, here within one process).  The summed M
equals the unsharded M within 1e-12, the run equals cp_arls_lev on the whole tensor
within 1e-10, and the fit from the summed terms equals cpa_fit's."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_16438_gb300 as cpa  # noqa: E402
from paper_2006_16438_gb300 import shard  # noqa: E402


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims,nnz,r,s,tau,nshards", [
    ((40, 30, 20, 12), 20000, 6, 3000, 1.0 / 3000, 2),
    ((60, 50, 40), 6000, 4, 1024, 1.0, 3),
])
def test_sharded_run_matches_unsharded(dims, nnz, r, s, tau, nshards):
    coo = synth.random_sparse_tensor(dims, nnz, seed=21)
    init = synth.gaussian_factors(dims, r, seed=22)
    bounds = shard.slice_bounds(coo.idx[0], dims[0], nshards)
    shards = [shard.shard_coo(coo, bounds, q) for q in range(nshards)]
    assert sum(c.nnz for c in shards) == coo.nnz
    whole = cpa.cpa_index_build(coo)
    parts = [cpa.cpa_index_build(c) for c in shards]
    fs = [torch.from_numpy(a).cuda() for a in init]
    a = shard.ShardedRun(parts, fs, rank=r, samples=s, tau=tau, seed=3)
    b = shard.ShardedRun([whole], fs, rank=r, samples=s, tau=tau, seed=3)
    # first update: same samples, summed partial M against the whole tensor's M
    ua = a.update(0, 0)
    ub = b.update(0, 0)
    assert ua["sbar"] == ub["sbar"]
    np.testing.assert_array_equal(ua["idx"].cpu().numpy(), ub["idx"].cpu().numpy())
    assert relerr(ua["M"].cpu().numpy(), ub["M"].cpu().numpy()) < 1e-12
    assert ua["nnz_sampled_local"] == ub["nnz_sampled_local"]
    for k in range(1, len(dims)):
        a.update(k, 0)
    a.it = 1
    a.iterate(2)
    ref = cpa.cp_arls_lev(whole, fs, rank=r, samples=s, tau=tau, iters=3, seed=3)
    for m in range(len(dims)):
        assert relerr(a.factors[m].cpu().numpy(), ref.factors[m].cpu().numpy()) < 1e-10
    assert relerr(a.lam.cpu().numpy(), ref.lam.cpu().numpy()) < 1e-10
    assert abs(a.fit() - ref.fit) < 1e-10
