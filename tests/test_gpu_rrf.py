"""Range-finder initialisation (App. F) on the GPU against the FP64 oracle.

The fibre draws are Philox integers (the same fibres on both sides); the sums are
FP64 atomic additions in an unfixed order, so each entry must match within 1e-12
of the sum of the absolute values of its terms (computed by the oracle from |X|
and |Omega|).
"""
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


def _abs_coo(coo):
    return synth.Coo(coo.dims, coo.idx, np.abs(coo.vals.astype(np.float64)))


CASES = [
    ("small-3way", lambda: synth.small_planted_tensor(0), 1000, 4),
    ("ragged-4way", lambda: synth.random_sparse_tensor((37, 29, 41, 13), 20000, seed=3, positive=False), 3001, 25),
    ("f32-values", lambda: synth.random_sparse_tensor((31, 17, 23), 2500, seed=4).as_dtype(np.float32), 777, 33),
    ("rank-64", lambda: synth.random_sparse_tensor((40, 30, 20), 5000, seed=5), 500, 64),
    ("one-draw", lambda: synth.random_sparse_tensor((9, 8, 7), 50, seed=6), 1, 1),
]


@pytest.mark.parametrize("name,make,s_init,r", CASES, ids=[c[0] for c in CASES])
def test_rrf_matches_oracle(name, make, s_init, r):
    coo = make()
    X = cpa.cpa_index_build(coo, dtype=coo.vals.dtype)
    c64 = coo.as_dtype(np.float64)
    Xo = oracle.Index(c64)
    Xa = oracle.Index(_abs_coo(c64))
    g = np.random.default_rng(7)
    for k in range(coo.order):
        omega = g.standard_normal((s_init, r))
        got = cpa.cpa_rrf_init(X, k, torch.from_numpy(omega), seed=13).cpu().numpy()
        want = oracle.rrf_init(Xo, k, omega, seed=13)
        bound = oracle.rrf_init(Xa, k, np.abs(omega), seed=13)
        assert np.all(np.abs(got - want) <= 1e-12 * bound + 1e-300), (name, k)


def test_rrf_errors_and_use():
    coo = synth.small_planted_tensor(0)
    X = cpa.cpa_index_build(coo)
    for mode, s_init, r in ((3, 10, 4), (-1, 10, 4), (0, 0, 4), (0, 10, 65)):
        with pytest.raises(cpa.CpaError) as ei:
            cpa.cpa_rrf_init(X, mode, torch.zeros((s_init, r), dtype=torch.float64), seed=0)
        assert ei.value.code == binding.ERR_ARG
    # an RRF start runs through Alg. 3 like any other initial guess
    g = torch.Generator().manual_seed(0)
    init = [cpa.cpa_rrf_init(X, k, torch.randn((1000, 4), dtype=torch.float64, generator=g), seed=k)
            for k in range(3)]
    res = cpa.cp_arls_lev(X, init, rank=4, samples=1024, tau=1.0 / 1024, iters=10, seed=1)
    assert np.isfinite(res.fit) and res.fit > 0.0
