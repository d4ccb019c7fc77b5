"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer outputs (Philox words, CDFs, sampled keys and counts, index layout) and the
sampling weights must match bit for bit when both sides get the same inputs.  FP64
products and solves must match within 1e-12 relative (stage) and 1e-10 relative
(whole runs: factors), the tolerance stated for the FP64 path; the fit within 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_16438_gb300 as cpa  # noqa: E402
from paper_2006_16438_gb300 import binding  # noqa: E402


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np_u64(t):
    return t.cpu().numpy().astype(np.uint64)


# --------------------------------------------------------------------------- Philox
def test_philox_bit_exact():
    g = np.random.default_rng(0)
    ctr = g.integers(0, 2**64, size=(3000, 4), dtype=np.uint64)
    key = [int(g.integers(0, 2**63)), int(g.integers(0, 2**63))]
    out = np_u64(cpa.cpa_philox4x64(cu(ctr), key))
    for i in range(0, 3000, 97):
        np.testing.assert_array_equal(out[i], oracle.philox4x64_10(ctr[i], key))


# --------------------------------------------------------------------------- leverage
@pytest.mark.parametrize("n,r", [(1, 1), (5, 1), (50, 7), (1717, 25), (4097, 25), (300, 64), (64, 64)])
def test_leverage_vs_oracle(n, r):
    g = np.random.default_rng(n + r)
    A = g.standard_normal((n, r)) * np.exp(0.5 * g.standard_normal(r))
    lev_gpu, warn = cpa.cpa_leverage(cu(A))
    lev_ref, rank = oracle.leverage(A)
    assert warn == 0 and rank == min(n, r)
    if n >= r:
        assert relerr(lev_gpu.cpu().numpy(), lev_ref) < 1e-11


# From 65,536 rows on the Gram and the row forms run in float pairs on the FP32 pipe:
# the streaming Gram (r <= 28, tiles of 16 rows, ragged tails; 4 x 4 blocks for r = 1
# and 8, 5 x 5 with two rows per pass for r = 25) and the one-pair-per-thread kernel
# (CPA_GRAM_STREAM_FP64=0, and r = 29, 32, 40), each checked against the oracle's QR
# leverage and for bit-identical reruns.
@pytest.mark.parametrize("stream_gram", ["1", "0"])
@pytest.mark.parametrize("n,r", [(65536, 1), (70001, 8), (100003, 25), (70003, 28), (81920, 29), (66001, 32),
                                 (70000, 40)])
def test_leverage_many_rows_vs_oracle(n, r, stream_gram, monkeypatch):
    monkeypatch.setenv("CPA_GRAM_STREAM_FP64", stream_gram)
    g = np.random.default_rng(n + r)
    A = g.standard_normal((n, r)) * np.exp(0.5 * g.standard_normal(r))
    A[: n // 9] *= 7.0  # a block of heavy rows
    lev_gpu, warn = cpa.cpa_leverage(cu(A))
    lev_ref, rank = oracle.leverage(A)
    assert warn == 0 and rank == r
    assert relerr(lev_gpu.cpu().numpy(), lev_ref) < 1e-11
    lev_again, _ = cpa.cpa_leverage(cu(A))
    assert torch.equal(lev_gpu, lev_again)


def test_leverage_rank_deficient():
    g = np.random.default_rng(2)
    B = g.standard_normal((40, 3))
    A = np.hstack([B, B[:, :1] * 3.0, np.zeros((40, 1))])
    lev_gpu, warn = cpa.cpa_leverage(cu(A))
    lev_ref, rank = oracle.leverage(A)
    assert rank == 3 and warn & 2
    assert relerr(lev_gpu.cpu().numpy(), lev_ref) < 1e-10
    assert abs(lev_gpu.sum().item() - 3) < 1e-9


# --------------------------------------------------------------------------- CDF
@pytest.mark.parametrize("n,r", [(1, 1), (13, 3), (4095, 25), (4097, 25), (100000, 10)])
def test_cdf_bit_exact(n, r):
    g = np.random.default_rng(n)
    A = g.standard_normal((n, r))
    A[: max(1, n // 7)] *= 20
    if n > 20:
        A[5:9] = 0  # rows of zero leverage
    lev, _ = oracle.leverage(A)
    C, T, mq, nz = cpa.cpa_cdf(cu(lev), r)
    d = oracle.ModeDist(lev, r)
    np.testing.assert_array_equal(np_u64(C), d.C)
    assert (T, mq, nz) == (d.T, d.maxq, d.nnzq)


# --------------------------------------------------------------------------- sampling
def _levs(dims, r, seed, skew):
    g = np.random.default_rng(seed)
    out = []
    for n in dims:
        A = g.standard_normal((n, r))
        A[: max(1, n // 6)] *= skew
        out.append(oracle.leverage(A)[0])
    return out


SKRP_CASES = [
    # dims, r, s, tau, skew
    ([40], 3, 100, 1.0, 1.0),
    ([37, 29], 4, 5000, 1.0, 5.0),
    ([37, 29], 4, 5000, 1.0 / 5000, 8.0),
    ([23, 19, 31], 5, 4096, 1.0 / 4096, 10.0),
    ([23, 19, 31], 5, 9000, 2.0 ** -9, 10.0),
    ([9, 8, 7, 6], 3, 3000, 1.0 / 3000, 6.0),
    ([183, 24, 1140], 25, 2 ** 17, 2.0 ** -17, 4.0),
    ([5, 6], 2, 10, 0.0, 1.0),          # tau = 0: top-s of the deterministic set
    ([4, 5], 2, 64, 0.0, 1.0),          # tau = 0 and s >= N: all rows deterministic
    ([7, 5, 3, 2, 2], 2, 777, 2.0 ** -6, 3.0),
]


@pytest.mark.parametrize("case", range(len(SKRP_CASES)))
def test_skrp_lev_bit_exact(case):
    dims, r, s, tau, skew = SKRP_CASES[case]
    levs = _levs(dims, r, 100 + case, skew)
    seed, it, k = 1234 + case, 7, 2
    got = cpa.cpa_skrp_lev([cu(l) for l in levs], r, samples=s, tau=tau, seed=seed, it=it, mode_k=k)
    ref = oracle.skrp_lev([oracle.ModeDist(l, r) for l in levs], s, tau, seed, it, k)
    assert got["sbar"] == ref["sbar"] and got["sdet"] == ref["sdet"]
    assert got["pdet"] == ref["pdet"]
    assert got["attempts"] == ref["attempts"]
    np.testing.assert_array_equal(np_u64(got["idx"]), ref["idx"])
    np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
    np.testing.assert_array_equal(got["wgt"].cpu().numpy(), ref["wgt"])


def test_skrp_reject_limit():
    # four heavy multi-indices hold all but ~1e-12 of the probability and are
    # deterministic; the light ones stay random, so almost every draw is rejected
    lev = np.array([0.5, 0.5 - 1e-12, 1e-12])
    with pytest.raises(cpa.CpaError) as e:
        cpa.cpa_skrp_lev([cu(lev), cu(lev)], 1, samples=20, tau=1e-9, reject_cap=40)
    assert e.value.code == -5
    with pytest.raises(oracle.OracleError) as e2:
        oracle.skrp_lev([oracle.ModeDist(lev, 1)] * 2, 20, 1e-9, 0, 0, 0, reject_cap=40)
    assert e2.value.code == oracle.ERR_REJECT_LIMIT


def test_skrp_det_cap():
    levs = _levs([60, 60, 60], 2, 6, 1.0)
    with pytest.raises(cpa.CpaError) as e:
        cpa.cpa_skrp_lev([cu(l) for l in levs], 2, samples=1 << 20, tau=1e-12, det_cap=1000)
    assert e.value.code == -6


# --------------------------------------------------------------------------- index
INDEX_CASES = [
    ((9, 7, 5, 4), 400, 1),
    ((60, 50, 40), 5000, 2),
    ((183, 24, 1140, 1717), 30000, 3),
    ((3, 2), 6, 4),
    ((2_000_000, 1_500_000, 1_800_000), 20000, 5),  # (key, i_k) does not fit 64 bits
]


@pytest.mark.parametrize("case", range(len(INDEX_CASES)))
def test_index_bit_exact(case):
    dims, nnz, seed = INDEX_CASES[case]
    coo = synth.random_sparse_tensor(dims, nnz, seed=seed)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        keys, off, ik, val = cpa.cpa_index_export(gi, k)
        rk, roff, rik, rval = oi.export(k)
        np.testing.assert_array_equal(np_u64(keys), rk)
        np.testing.assert_array_equal(np_u64(off), roff.astype(np.uint64))
        np.testing.assert_array_equal(ik.cpu().numpy(), rik)
        np.testing.assert_array_equal(val.cpu().numpy(), rval)


def test_index_errors():
    coo = synth.random_sparse_tensor((5, 4, 3), 20, seed=1)
    bad = synth.Coo(coo.dims, [c.copy() for c in coo.idx], coo.vals)
    bad.idx[1][3] = 4
    with pytest.raises(cpa.CpaError) as e:
        cpa.cpa_index_build(bad)
    assert e.value.code == -2
    dup = synth.Coo(coo.dims, [np.append(c, c[0]) for c in coo.idx], np.append(coo.vals, 1.0))
    with pytest.raises(cpa.CpaError) as e:
        cpa.cpa_index_build(dup)
    assert e.value.code == -3


def test_index_empty_tensor():
    coo = synth.Coo((4, 5, 6), [np.zeros(0, np.int32)] * 3, np.zeros(0))
    gi = cpa.cpa_index_build(coo)
    assert gi.nfib(0) == 0


# --------------------------------------------------------------------------- products
def _sample_for(coo, facs, k, r, s, tau, seed=3):
    others = [m for m in range(len(coo.dims)) if m != k]
    ds = [oracle.ModeDist(oracle.leverage(facs[m])[0], r) for m in others]
    return oracle.skrp_lev(ds, s, tau, seed, 0, k)


@pytest.mark.parametrize("dims,nnz,r,s,tau", [
    ((30, 20, 25), 3000, 5, 2000, 1.0),
    ((30, 20, 25), 3000, 5, 2000, 1 / 2000),
    ((183, 24, 1140, 1717), 200000, 25, 2 ** 14, 2.0 ** -14),
    ((50, 40, 30), 20000, 40, 5000, 1.0),    # r > 32: two columns per lane
    ((500, 300, 200), 100000, 8, 20000, 1.0),  # M too large for shared memory
])
def test_sampled_mttkrp_vs_oracle(dims, nnz, r, s, tau):
    coo = synth.random_sparse_tensor(dims, nnz, seed=9)
    facs = synth.gaussian_factors(dims, r, seed=2)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        smp = _sample_for(coo, facs, k, r, s, tau)
        M, G, nz = cpa.cpa_sampled_mttkrp(gi, k, [cu(f) for f in facs], cu(smp["idx"]), cu(smp["wgt"]))
        Mr, Gr, nzr = oracle.sampled_mttkrp(oi, k, facs, smp["idx"], smp["wgt"])
        assert nz == nzr
        assert relerr(M.cpu().numpy(), Mr) < 1e-12
        assert relerr(G.cpu().numpy(), Gr) < 1e-12


def test_sampled_mttkrp_empty_fibres_and_heavy_fibre():
    # one fibre with many nonzeros (spans several warp chunks) and keys with no nonzeros
    dims = (5000, 3, 2)
    n = 4000
    idx = [np.arange(n, dtype=np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)]
    coo = synth.Coo(dims, idx, np.linspace(0.5, 1.5, n))
    facs = synth.gaussian_factors(dims, 6, seed=4)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    keys = np.array([0, 1, 2, 3, 4, 5], dtype=np.uint64)  # only key 0 has a fibre
    w = np.array([1.5, 0.5, 2.0, 1.0, 1.0, 3.0])
    M, G, nz = cpa.cpa_sampled_mttkrp(gi, 0, [cu(f) for f in facs], cu(keys), cu(w))
    Mr, Gr, nzr = oracle.sampled_mttkrp(oi, 0, facs, keys, w)
    assert nz == nzr == n
    assert relerr(M.cpu().numpy(), Mr) < 1e-12 and relerr(G.cpu().numpy(), Gr) < 1e-12


@pytest.mark.parametrize("slab_bytes", [64, 4096])
@pytest.mark.parametrize("dims,nnz,r,s,tau", [
    ((300, 20, 25), 30000, 5, 2000, 1.0),
    ((3000, 4, 5), 20000, 25, 500, 1.0),      # fibres of about 1000 nonzeros: heavy slab ranges
    ((183, 24, 1140, 1717), 200000, 25, 2 ** 14, 2.0 ** -14),
    ((500, 40, 30), 20000, 40, 5000, 1.0),    # r > 32: two columns per lane
    ((20000, 30, 40), 200000, 25, 4000, 1.0),
])
def test_sampled_mttkrp_row_slabs_vs_oracle(monkeypatch, slab_bytes, dims, nnz, r, s, tau):
    """The row-slab path (M accumulated one slab of rows at a time, every fibre cut at
    the slab boundaries of its sorted i_k), forced at these sizes by a small slab."""
    monkeypatch.setenv("CPA_MTTKRP_SLAB_BYTES", str(slab_bytes))
    coo = synth.random_sparse_tensor(dims, nnz, seed=9)
    facs = synth.gaussian_factors(dims, r, seed=2)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    for k in range(len(dims)):
        smp = _sample_for(coo, facs, k, r, s, tau)
        M, G, nz = cpa.cpa_sampled_mttkrp(gi, k, [cu(f) for f in facs], cu(smp["idx"]), cu(smp["wgt"]))
        Mr, Gr, nzr = oracle.sampled_mttkrp(oi, k, facs, smp["idx"], smp["wgt"])
        assert nz == nzr
        assert relerr(M.cpu().numpy(), Mr) < 1e-12
        assert relerr(G.cpu().numpy(), Gr) < 1e-12


def test_row_slabs_skewed(monkeypatch):
    """A Zipf-skewed planted tensor whose first mode has 30,000 rows, its M in row
    slabs: long fibres are cut into pieces shared by the blocks; FP64 products equal
    the oracle's, and a mixed-precision run works."""
    monkeypatch.setenv("CPA_MTTKRP_SLAB_BYTES", "100000")
    coo = synth.planted_cp_tensor((30000, 60, 50), 5, events=300000, seed=3, zipf_alpha=1.1)
    facs = synth.gaussian_factors(coo.dims, 5, seed=4)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    smp = _sample_for(coo, facs, 0, 5, 2000, 1.0 / 2000)
    M, G, nz = cpa.cpa_sampled_mttkrp(gi, 0, [cu(f) for f in facs], cu(smp["idx"]), cu(smp["wgt"]))
    Mr, Gr, nzr = oracle.sampled_mttkrp(oi, 0, facs, smp["idx"], smp["wgt"])
    assert nz == nzr and nz > 0
    assert relerr(M.cpu().numpy(), Mr) < 1e-12
    res = cpa.cp_arls_lev(gi, [cu(a) for a in facs], rank=5, samples=2000, tau=1.0 / 2000, iters=3,
                          precision=binding.MIXED)
    assert np.isfinite(res.fit)


def test_whole_run_row_slabs(monkeypatch):
    """Alg. 3 with every mode's M in row slabs (FP64: factors within 1e-10 of the
    oracle; mixed precision runs)."""
    monkeypatch.setenv("CPA_MTTKRP_SLAB_BYTES", "256")
    coo = synth.small_planted_tensor(0)
    _compare_run(coo, 4, 1024, 1.0 / 1024, 5)
    gi = cpa.cpa_index_build(coo)
    init = synth.gaussian_factors(coo.dims, 4, seed=0)
    res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=4, samples=1024, tau=1.0 / 1024, iters=5,
                          precision=binding.MIXED)
    assert np.isfinite(res.fit)


def test_solve_vs_oracle():
    g = np.random.default_rng(7)
    for n, r in [(1, 1), (183, 25), (5000, 25), (77, 64)]:
        B = g.standard_normal((3 * r + 5, r))
        G = B.T @ B
        M = g.standard_normal((n, r))
        A, lam, warn = cpa.cpa_solve(cu(G), cu(M))
        Ar, rc = oracle.solve(G, M)
        An, lamr = oracle.normalize(Ar)
        assert warn == 0 and rc == 0
        assert relerr(lam.cpu().numpy(), lamr) < 1e-12
        assert relerr(A.cpu().numpy(), An) < 1e-11
    Gs = G.copy()
    Gs[:, 3] = 0
    Gs[3, :] = 0
    A, lam, warn = cpa.cpa_solve(cu(Gs), cu(M))
    Ar, rc = oracle.solve(Gs, M)
    An, lamr = oracle.normalize(Ar)
    assert warn & 1 and rc == 1
    assert relerr(A.cpu().numpy(), An) < 1e-9


@pytest.mark.parametrize("r,deficit", [(2, 1), (7, 3), (25, 5), (50, 2), (64, 9)])
def test_singular_solve_pinv_vs_oracle(r, deficit):
    """A rank-deficient sampled Gram takes the pseudo-inverse path (block-parallel
    Jacobi on the GPU, serial Jacobi in the oracle): the same pinv solution and the
    singular-Gram warning on both sides."""
    g = np.random.default_rng(100 + r)
    B = g.standard_normal((r, r - deficit)) * np.exp(g.standard_normal(r - deficit))
    G = B @ B.T
    M = g.standard_normal((40, r)) @ (G + np.eye(r) * 0.0)  # right-hand sides in range(G)
    A, lam, warn = cpa.cpa_solve(cu(G), cu(M))
    Ar, rc = oracle.solve(G, M)
    An, lamr = oracle.normalize(Ar)
    assert warn & 1 and rc & 1
    assert relerr(A.cpu().numpy(), An) < 1e-9
    assert relerr(lam.cpu().numpy(), lamr) < 1e-9


def test_fit_vs_oracle():
    for dims, nnz in [((30, 20, 25), 3000), ((183, 24, 114, 171), 50000)]:
        coo = synth.random_sparse_tensor(dims, nnz, seed=11)
        facs = synth.gaussian_factors(dims, 7, seed=3)
        lam = np.linspace(0.5, 2.0, 7)
        gi = cpa.cpa_index_build(coo)
        oi = oracle.Index(coo)
        f = cpa.cpa_fit(gi, [cu(a) for a in facs], cu(lam))
        fr = oracle.fit(oi, facs, lam)
        assert abs(f - fr) < 1e-10


# --------------------------------------------------------------------------- whole runs
def _compare_run(coo, r, s, tau, iters, seed=0, init_seed=0, tol_f=1e-10, dist=0):
    init = synth.gaussian_factors(coo.dims, r, seed=init_seed)
    gi = cpa.cpa_index_build(coo)
    res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=seed,
                          distribution=dist)
    oi = oracle.Index(coo)
    lam, fs, fit, done, warn = oracle.cp_arls_lev(oi, init, rank=r, samples=s, tau=tau, iters=iters,
                                                  seed=seed, distribution=dist)
    errs = [relerr(a.cpu().numpy(), b) for a, b in zip(res.factors, fs)]
    assert max(errs) < tol_f, errs
    assert relerr(res.lam.cpu().numpy(), lam) < tol_f
    assert abs(res.fit - fit) < 1e-10
    return res, fit


def test_small_planted_random_sampling_10_iters():
    """60x50x40 planted tensor, r = 4, s = 1024, random sampling, 10 iterations."""
    coo = synth.small_planted_tensor(0)
    res, fit = _compare_run(coo, 4, 1024, 1.0, 10)
    assert res.stats["mode_updates"] == 30


def test_small_planted_hybrid():
    coo = synth.small_planted_tensor(0)
    res, fit = _compare_run(coo, 4, 1024, 1.0 / 1024, 5)
    assert res.stats["sdet_last"] > 0


@pytest.mark.parametrize("dist", [oracle.DIST_UNIFORM, oracle.DIST_LENGTH_SQUARED])
@pytest.mark.parametrize("tau", [1.0, 1.0 / 1024])
def test_app_b_distributions_whole_run(dist, tau):
    """Uniform and length-squared sampling (App. B) through the whole of Alg. 3, random
    and hybrid, on the small planted tensor and a ragged 4-way tensor."""
    _compare_run(synth.small_planted_tensor(0), 4, 1024, tau, 6, dist=dist)
    _compare_run(synth.random_sparse_tensor((37, 29, 41, 13), 20000, seed=3), 6, 3000, tau, 3, dist=dist)


@pytest.mark.parametrize("dims,nnz,r,s", [((37, 29, 41, 13), 20000, 6, 3000), ((40, 30, 20), 8000, 3, 500),
                                          ((30, 4, 20), 1500, 5, 400)])  # n_1 < r: rank-deficient factor
def test_ragged_runs(dims, nnz, r, s):
    coo = synth.random_sparse_tensor(dims, nnz, seed=5)
    _compare_run(coo, r, s, 1.0 / s, 3, seed=9)


def test_all_rows_deterministic_is_cp_als():
    """tau = 0, s >= N: every update is the exact CP-ALS update (Eq. 1.1)."""
    coo = synth.random_sparse_tensor((8, 7, 6), 150, seed=8)
    r = 3
    init = synth.gaussian_factors(coo.dims, r, seed=1)
    gi = cpa.cpa_index_build(coo)
    res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=64, tau=0.0, iters=4)
    oi = oracle.Index(coo)
    lam, fs, fit, _ = oracle.cp_als(oi, init, rank=r, iters=4)
    assert max(relerr(a.cpu().numpy(), b) for a, b in zip(res.factors, fs)) < 1e-9
    assert abs(res.fit - fit) < 1e-9


def test_host_coo_entry_point():
    coo = synth.small_planted_tensor(1)
    init = synth.gaussian_factors(coo.dims, 4, seed=2)
    res = cpa.cp_arls_lev_coo(coo, init, rank=4, samples=1024, tau=1.0, iters=3, seed=4)
    oi = oracle.Index(coo)
    lam, fs, fit, _, _ = oracle.cp_arls_lev(oi, init, rank=4, samples=1024, tau=1.0, iters=3, seed=4)
    assert max(relerr(a, b) for a, b in zip(res.factors, fs)) < 1e-10
    assert abs(res.fit - fit) < 1e-10


@pytest.mark.slow
def test_uber_shaped_full_size_one_iteration():
    """The 183x24x1140x1717 planted tensor (3.3M nonzeros), r = 25, s = 2^17,
    tau = 2^-17: one outer iteration (4 mode updates) against the oracle."""
    coo = synth.uber_like_tensor(0)
    res, fit = _compare_run(coo, 25, 2 ** 17, 2.0 ** -17, 1)
    assert res.stats["nnz_sampled_total"] > 0
