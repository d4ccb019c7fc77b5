"""Full CP-ALS on the GPU (exact MTTKRP over the fibre index, Hadamard-of-Grams
normal equations) against the oracle's CP-ALS from the same initial factors:
factors within 1e-10 relative and the fit within 1e-10 in FP64; the mixed-precision
run converges to the same fit on an exactly low-rank tensor."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_16438_gb300 as cpa  # noqa: E402
from paper_2006_16438_gb300 import binding  # noqa: E402


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims,nnz,r,iters", [((30, 20, 25), 2000, 4, 3), ((13, 17, 11, 9), 3000, 6, 2),
                                              ((60, 50, 40), 4000, 25, 2)])
def test_cp_als_matches_oracle(dims, nnz, r, iters):
    coo = synth.random_sparse_tensor(dims, nnz, seed=3)
    init = synth.gaussian_factors(dims, r, seed=4)
    gi = cpa.cpa_index_build(coo)
    got = cpa.cp_als(gi, [torch.from_numpy(a).cuda() for a in init], rank=r, iters=iters)
    lam, fs, fit, _ = oracle.cp_als(oracle.Index(coo), init, rank=r, iters=iters)
    for m in range(len(dims)):
        assert relerr(got.factors[m].cpu().numpy(), fs[m]) < 1e-10
    assert relerr(got.lam.cpu().numpy(), lam) < 1e-10
    assert abs(got.fit - fit) < 1e-10


def test_cp_als_mixed_reaches_planted_fit():
    coo, _, _ = synth.exact_lowrank_tensor((30, 25, 20), 3, seed=4, density=0.6)
    init = synth.gaussian_factors(coo.dims, 3, seed=1)
    gi = cpa.cpa_index_build(coo)
    f64 = cpa.cp_als(gi, [torch.from_numpy(a).cuda() for a in init], rank=3, iters=100)
    mix = cpa.cp_als(gi, [torch.from_numpy(a).cuda() for a in init], rank=3, iters=100,
                     precision=binding.MIXED)
    assert f64.fit > 1 - 1e-6
    assert abs(mix.fit - f64.fit) < 1e-3
