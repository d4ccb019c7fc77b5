"""One mode update through cpa_mode_update, FP64 and mixed precision.

FP64: the rows and counts equal the oracle's bit for bit; the weights agree to
1e-13 relative (they are bit-exact only when both sides start from the same leverage
vectors, which the stage tests check: here the GPU's Cholesky leverage and the
oracle's QR leverage differ in the last bits); the new factor matches within 1e-10
relative.  Mixed precision (FP32 products, FP64 factorisations):
the leverage scores come from FP32 Grams, so the rows may differ from the FP64
oracle's; the check feeds the GPU's own rows to the oracle's FP64 sampled MTTKRP and
solve and requires the factor within 2e-4 relative, the tolerance stated for the
mixed path.
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
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


CASES = [
    ((60, 50, 40), 4000, 4, 1024, 1.0 / 1024),
    ((37, 29, 41, 13), 20000, 6, 3000, 1.0),
    ((183, 24, 1140, 1717), 200000, 25, 2 ** 14, 2.0 ** -14),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mode_update_fp64_matches_oracle(case):
    dims, nnz, r, s, tau = CASES[case]
    coo = synth.random_sparse_tensor(dims, nnz, seed=case + 1)
    facs = synth.gaussian_factors(dims, r, seed=case + 2)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=s, tau=tau, seed=7, it=3)
        ref = oracle.mode_update(oi, facs, k, rank=r, samples=s, tau=tau, seed=7, it=3)
        assert got["sbar"] == ref["sbar"] and got["sdet"] == ref["sdet"]
        assert abs(got["pdet"] - ref["pdet"]) <= 1e-13 * max(ref["pdet"], 1e-300)
        np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), ref["idx"])
        np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
        assert relerr(got["wgt"].cpu().numpy(), ref["wgt"]) < 1e-13
        assert relerr(fs[k].cpu().numpy(), ref["A"]) < 1e-10
        assert relerr(got["lam"].cpu().numpy(), ref["lam"]) < 1e-10


@pytest.mark.parametrize("dist", [binding.DIST_UNIFORM, binding.DIST_LENGTH_SQUARED])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_mode_update_app_b_matches_oracle(case, dist):
    """Uniform and length-squared sampling (App. B): rows and counts bit-exact (the
    uniform scores are the same two IEEE operations on both sides; length-squared
    scores agree to the last bits), weights to 1e-13, the new factor to 1e-10."""
    dims, nnz, r, s, tau = CASES[case]
    coo = synth.random_sparse_tensor(dims, nnz, seed=case + 1)
    facs = synth.gaussian_factors(dims, r, seed=case + 2)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=s, tau=tau, seed=7, it=3, distribution=dist)
        ref = oracle.mode_update(oi, facs, k, rank=r, samples=s, tau=tau, seed=7, it=3, distribution=dist)
        assert got["sbar"] == ref["sbar"] and got["sdet"] == ref["sdet"]
        np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), ref["idx"])
        np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
        assert relerr(got["wgt"].cpu().numpy(), ref["wgt"]) < 1e-13
        assert relerr(fs[k].cpu().numpy(), ref["A"]) < 1e-10


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mode_update_mixed_within_2e4(case):
    dims, nnz, r, s, tau = CASES[case]
    coo = synth.random_sparse_tensor(dims, nnz, seed=case + 1)
    facs = synth.gaussian_factors(dims, r, seed=case + 2)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=s, tau=tau, seed=7, it=3,
                                  precision=binding.MIXED)
        idx = got["idx"].cpu().numpy().astype(np.uint64)
        wgt = got["wgt"].cpu().numpy()
        M, G, _ = oracle.sampled_mttkrp(oi, k, facs, idx, wgt)
        A, _ = oracle.solve(G, M)
        An, lam = oracle.normalize(A)
        assert relerr(fs[k].cpu().numpy(), An) < 2e-4
        assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4
        # the sampled rows are valid: same count of rows as weights, positive weights
        assert got["sbar"] == idx.size and np.all(wgt > 0)


def test_mixed_run_reaches_planted_fit():
    """Exact low-rank tensor: the mixed path converges like the FP64 path.  Its fit is
    evaluated as ||X||^2 - 2<X,M> + ||M||^2 with FP32 products, so near fit = 1 it
    resolves only about sqrt(2^-24) ~ 3e-4 (the FP64 floor is 1.5e-8)."""
    coo, lam0, f0 = synth.exact_lowrank_tensor((30, 25, 20), 3, seed=4, density=0.6)
    init = synth.gaussian_factors(coo.dims, 3, seed=1)
    gi = cpa.cpa_index_build(coo)
    f64 = cpa.cp_arls_lev(gi, [torch.from_numpy(a).cuda() for a in init], rank=3, samples=500, tau=1.0,
                          iters=150, seed=2)
    mix = cpa.cp_arls_lev(gi, [torch.from_numpy(a).cuda() for a in init], rank=3, samples=500, tau=1.0,
                          iters=150, seed=2, precision=binding.MIXED)
    assert f64.fit > 1 - 1e-6
    assert mix.fit > 1 - 1e-3
    assert abs(mix.fit - f64.fit) < 1e-3


def test_mixed_small_planted_fit_close_to_fp64():
    coo = synth.small_planted_tensor(0)
    init = synth.gaussian_factors(coo.dims, 4, seed=0)
    gi = cpa.cpa_index_build(coo)
    f64 = cpa.cp_arls_lev(gi, [torch.from_numpy(a).cuda() for a in init], rank=4, samples=1024, tau=1.0,
                          iters=10, seed=0)
    mix = cpa.cp_arls_lev(gi, [torch.from_numpy(a).cuda() for a in init], rank=4, samples=1024, tau=1.0,
                          iters=10, seed=0, precision=binding.MIXED)
    assert abs(mix.fit - f64.fit) < 1e-2


def test_epoch_graph_keyed_by_fit_mode():
    """The one-graph call is cached per (iterations, fit): a call with the fit after
    one without it (same index, same options otherwise) still computes the fit."""
    coo = synth.small_planted_tensor(0)
    init = synth.gaussian_factors(coo.dims, 4, seed=0)
    gi = cpa.cpa_index_build(coo)
    a = cpa.cp_arls_lev(gi, [torch.from_numpy(x).cuda() for x in init], rank=4, samples=1024, tau=1.0, iters=2,
                        seed=0, fit_mode=binding.FIT_NONE)
    assert np.isnan(a.fit)
    b = cpa.cp_arls_lev(gi, [torch.from_numpy(x).cuda() for x in init], rank=4, samples=1024, tau=1.0, iters=2,
                        seed=0, fit_mode=binding.FIT_EXACT)
    c = cpa.cp_arls_lev(cpa.cpa_index_build(coo), [torch.from_numpy(x).cuda() for x in init], rank=4,
                        samples=1024, tau=1.0, iters=2, seed=0)
    assert np.isfinite(b.fit) and abs(b.fit - c.fit) < 1e-12


@pytest.mark.parametrize("r", [8, 25])
def test_mixed_float_pair_leverage_matches_fp64_rows(monkeypatch, r):
    """Mixed precision with factors that are exact in FP32 and a first mode of 70,000
    rows: the factor Gram (k_gram_rows_ff) and the leverage rows (k_lev_rows_ff) of
    the FP32 factors run in float-pair arithmetic (about 2^-44), so the leverage
    distributions, and with them the sampled rows and counts, equal the FP64
    oracle's; weights to 1e-12."""
    monkeypatch.setenv("CPA_LEV_FLOAT_PAIR", "1")  # the float-pair kernels instead of the tensor cores
    dims = (70000, 40, 30)
    coo = synth.random_sparse_tensor(dims, 300000, seed=11)
    facs = [a.astype(np.float32).astype(np.float64) for a in synth.gaussian_factors(dims, r, seed=12)]
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in (1, 2):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=4000, tau=1.0 / 4000, seed=5, it=1,
                                  precision=binding.MIXED)
        ref = oracle.mode_update(oi, facs, k, rank=r, samples=4000, tau=1.0 / 4000, seed=5, it=1)
        assert got["sbar"] == ref["sbar"] and got["sdet"] == ref["sdet"]
        np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), ref["idx"])
        np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
        assert relerr(got["wgt"].cpu().numpy(), ref["wgt"]) < 1e-12


@pytest.mark.parametrize("r", [33, 40, 64])
def test_mode_update_mixed_wide_rank_within_2e4(r):
    """Mixed precision with r > 32 (the tensor-core sampled Gram with N = 64): the
    new factor within 2e-4 of the FP64 oracle's solve on the GPU's own rows."""
    dims = (50, 40, 30)
    coo = synth.random_sparse_tensor(dims, 20000, seed=r)
    facs = synth.gaussian_factors(dims, r, seed=r + 1)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(3):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=1200, tau=1.0, seed=3, it=0, precision=binding.MIXED)
        idx = got["idx"].cpu().numpy().astype(np.uint64)
        wgt = got["wgt"].cpu().numpy()
        M, G, _ = oracle.sampled_mttkrp(oi, k, facs, idx, wgt)
        A, _ = oracle.solve(G, M)
        An, lam = oracle.normalize(A)
        assert relerr(fs[k].cpu().numpy(), An) < 2e-4
        assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4


@pytest.mark.parametrize("r", [4, 25, 40, 64])
def test_mode_update_mixed_tensor_core_gram(monkeypatch, r):
    """The sampled Gram on the tensor cores (CPA_GRAM_TENSOR_CORES=1: tcgen05 kind::tf32
    with the three-product split, M = 128, N = 32 or 64): the new factor within 2e-4
    of the FP64 oracle's solve on the GPU's own rows."""
    monkeypatch.setenv("CPA_GRAM_TENSOR_CORES", "1")
    dims = (50, 40, 30)
    coo = synth.random_sparse_tensor(dims, 20000, seed=100 + r)
    facs = synth.gaussian_factors(dims, r, seed=r + 3)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(3):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=1500, tau=1.0, seed=4, it=0, precision=binding.MIXED)
        idx = got["idx"].cpu().numpy().astype(np.uint64)
        wgt = got["wgt"].cpu().numpy()
        M, G, _ = oracle.sampled_mttkrp(oi, k, facs, idx, wgt)
        A, _ = oracle.solve(G, M)
        An, lam = oracle.normalize(A)
        assert relerr(fs[k].cpu().numpy(), An) < 2e-4


@pytest.mark.parametrize("r", [8, 25, 40, 64])
def test_mode_update_mixed_many_rows_within_2e4(r):
    """Mixed precision on a mode of 70,000 rows: the solve A = M G^-1 runs one
    thread per row (k_solve_rows_f32, the row and its sums in registers); the new
    factor within 2e-4 of the FP64 oracle's solve on the GPU's own rows."""
    dims = (70000, 40, 30)
    coo = synth.random_sparse_tensor(dims, 300000, seed=20 + r)
    facs = synth.gaussian_factors(dims, r, seed=r + 5)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    fs = [torch.from_numpy(a).cuda() for a in facs]
    got = cpa.cpa_mode_update(gi, fs, 0, rank=r, samples=3000, tau=1.0, seed=6, it=0, precision=binding.MIXED)
    idx = got["idx"].cpu().numpy().astype(np.uint64)
    wgt = got["wgt"].cpu().numpy()
    M, G, _ = oracle.sampled_mttkrp(oi, 0, facs, idx, wgt)
    A, _ = oracle.solve(G, M)
    An, lam = oracle.normalize(A)
    assert relerr(fs[0].cpu().numpy(), An) < 2e-4
    assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4


@pytest.mark.parametrize("r", [8, 25, 40])
def test_mixed_tensor_core_leverage_close_to_fp64(r):
    """Mixed precision on a first mode of 70,000 rows: its factor Gram and leverage
    rows run on the tensor cores (tcgen05 kind::tf32, three-product hi/lo split, about
    FP32 accuracy), so the sampling distribution of that mode is the FP64 one to about
    1e-6 relative.  Updates of the other modes sample from it: nearly all of the FP64
    oracle's rows are drawn (a draw flips only where a CDF boundary moved past it), the
    weights of the common rows agree within 1e-4 and the new factor is within 2e-4 of the
    oracle's solve on the GPU's own rows."""
    dims = (70000, 40, 30)
    coo = synth.random_sparse_tensor(dims, 300000, seed=13 + r)
    facs = synth.gaussian_factors(dims, r, seed=14 + r)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in (1, 2):
        fs = [torch.from_numpy(a).cuda() for a in facs]
        got = cpa.cpa_mode_update(gi, fs, k, rank=r, samples=4000, tau=1.0 / 4000, seed=5, it=1,
                                  precision=binding.MIXED)
        ref = oracle.mode_update(oi, facs, k, rank=r, samples=4000, tau=1.0 / 4000, seed=5, it=1)
        gidx = got["idx"].cpu().numpy().astype(np.uint64)
        gw = got["wgt"].cpu().numpy()
        common, gi_pos, ri_pos = np.intersect1d(gidx, ref["idx"], return_indices=True)
        assert common.size >= 0.95 * ref["idx"].size
        assert relerr(gw[gi_pos], ref["wgt"][ri_pos]) < 1e-4
        M, G, _ = oracle.sampled_mttkrp(oi, k, facs, gidx, gw)
        A, _ = oracle.solve(G, M)
        An, lam = oracle.normalize(A)
        assert relerr(fs[k].cpu().numpy(), An) < 2e-4
        assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4



@pytest.mark.gpu
@pytest.mark.parametrize("r", [8, 25, 30])
def test_mixed_refresh_of_folded_mode(r):
    """A mixed-precision update of a 70,000-row mode: the solve is folded into the
    sampled MTTKRP, and the refresh streams the unnormalised rows (row stride r rounded
    up to 4 floats) through the FP32-pipe Gram and the tensor-core row forms, which
    write the normalised factor.  The factor and lambda are within 2e-4 of the FP64
    oracle's solve on the GPU's own sampled rows."""
    dims = (70000, 40, 30)
    coo = synth.random_sparse_tensor(dims, 300000, seed=31 + r)
    facs = synth.gaussian_factors(dims, r, seed=32 + r)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    fs = [torch.from_numpy(a).cuda() for a in facs]
    got = cpa.cpa_mode_update(gi, fs, 0, rank=r, samples=4000, tau=1.0 / 4000, seed=5, it=1,
                              precision=binding.MIXED)
    idx = got["idx"].cpu().numpy().astype(np.uint64)
    wgt = got["wgt"].cpu().numpy()
    M, G, _ = oracle.sampled_mttkrp(oi, 0, facs, idx, wgt)
    A, _ = oracle.solve(G, M)
    An, lam = oracle.normalize(A)
    assert relerr(fs[0].cpu().numpy(), An) < 2e-4
    assert relerr(got["lam"].cpu().numpy(), lam) < 2e-4