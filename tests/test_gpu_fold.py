"""The update with the normal-equation solve folded into the sampled MTTKRP.

For modes of at least 65,536 rows (CPA_FOLD_ROWS; the tests lower it to fold every
mode) the update forms the sampled Gram first, factors it, and accumulates
A_k = X~_(k) (U~ G~^-1) directly: the same least-squares solution as M G~^-1 of
Alg. 3 without the n_k r^2 row solve.  FP64 runs must match the FP64 oracle within
1e-10 (with the reproducible sorted MTTKRP and with FP64 atomics); FP32 runs
(16-byte atomics into rows padded to a multiple of 4 floats) within 2e-4 of the
oracle's solve on the GPU's own rows.
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


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare_run(coo, r, s, tau, iters, seed=0):
    init = synth.gaussian_factors(coo.dims, r, seed=1)
    gi = cpa.cpa_index_build(coo)
    res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=seed)
    oi = oracle.Index(coo)
    lam, fs, fit, _, _ = oracle.cp_arls_lev(oi, init, rank=r, samples=s, tau=tau, iters=iters, seed=seed)
    errs = [relerr(a.cpu().numpy(), b) for a, b in zip(res.factors, fs)]
    assert max(errs) < 1e-10, errs
    assert relerr(res.lam.cpu().numpy(), lam) < 1e-10
    assert abs(res.fit - fit) < 1e-10


@pytest.mark.parametrize("det", ["1", "0"])
@pytest.mark.parametrize("slab_bytes", [None, "1024"])
def test_folded_fp64_runs_match_oracle(monkeypatch, det, slab_bytes):
    """Every mode folded; the MTTKRP reproducible (sorted) or with FP64 atomics, in one
    pass or in row slabs of 1 KB (several slabs, each pass adding its own rows)."""
    monkeypatch.setenv("CPA_FOLD_ROWS", "1")
    monkeypatch.setenv("CPA_DET_MTTKRP", det)
    if slab_bytes:
        monkeypatch.setenv("CPA_MTTKRP_SLAB_BYTES", slab_bytes)
    _compare_run(synth.small_planted_tensor(0), 4, 1024, 1.0 / 1024, 5)
    _compare_run(synth.random_sparse_tensor((37, 29, 41, 13), 20000, seed=3), 6, 3000, 1.0, 3)
    _compare_run(synth.random_sparse_tensor((50, 40, 30), 20000, seed=4), 40, 4000, 1.0 / 4000, 2)


@pytest.mark.parametrize("r", [4, 25, 40, 64])
@pytest.mark.parametrize("slab_bytes", [None, "2048"])
def test_folded_mixed_update_within_2e4(monkeypatch, r, slab_bytes):
    """FP32 folded updates (rows of r rounded up to 4 floats, 16-byte atomics, one or
    two float4 pieces per lane): the new factor and lambda within 2e-4 of the FP64
    oracle's solve on the GPU's own sampled rows."""
    monkeypatch.setenv("CPA_FOLD_ROWS", "1")
    if slab_bytes:
        monkeypatch.setenv("CPA_MTTKRP_SLAB_BYTES", slab_bytes)
    dims = (50, 40, 30)
    coo = synth.random_sparse_tensor(dims, 20000, seed=200 + r)
    facs = synth.gaussian_factors(dims, r, seed=r + 7)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(3):
        fs = [cu(a) for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=1500, tau=1.0 / 1500, seed=4, it=0,
                                  precision=binding.MIXED)
        idx = got["idx"].cpu().numpy().astype(np.uint64)
        wgt = got["wgt"].cpu().numpy()
        M, G, _ = oracle.sampled_mttkrp(oi, k, facs, idx, wgt)
        A, _ = oracle.solve(G, M)
        An, lam = oracle.normalize(A)
        assert relerr(fs[k].cpu().numpy(), An) < 2e-4
        assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4


def test_folded_mode_of_many_rows_fp64(monkeypatch):
    """The default threshold: a 70,000-row mode is folded, the others are not; one
    FP64 update of each mode against the oracle (rows bit-exact, factor 1e-10)."""
    monkeypatch.delenv("CPA_FOLD_ROWS", raising=False)
    dims, r, s = (70000, 40, 30), 8, 3000
    coo = synth.random_sparse_tensor(dims, 300000, seed=77)
    facs = synth.gaussian_factors(dims, r, seed=78)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(3):
        fs = [cu(a) for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=s, tau=1.0 / s, seed=2, it=1)
        ref = oracle.mode_update(oi, facs, k, rank=r, samples=s, tau=1.0 / s, seed=2, it=1)
        np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), ref["idx"])
        np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
        assert relerr(fs[k].cpu().numpy(), ref["A"]) < 1e-10
        assert relerr(got["lam"].cpu().numpy(), ref["lam"]) < 1e-10
