"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Every check here compares the oracle with something other than itself: numpy's own
Philox generator, SVD leverage scores, explicit Khatri-Rao products, brute-force
enumeration, math.fsum, dense unfoldings, least squares by numpy, closed forms and
the sizes printed in the paper.  None of these tests need a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from tests import _ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def test_philox_matches_numpy(orc):
    g = np.random.default_rng(1)
    for _ in range(50):
        ctr = g.integers(0, 2**63, size=4, dtype=np.uint64)
        ctr[0] |= np.uint64(1)
        key = g.integers(0, 2**63, size=2, dtype=np.uint64)
        np.testing.assert_array_equal(orc.philox4x64_10(ctr, key), _ref.numpy_philox_block(ctr, key))
    # counters that exercise the carry between words in numpy's increment
    for ctr in ([0, 1, 0, 0], [0, 0, 0, 7], [5, 0, 1 << 32, 9]):
        key = [3, 0]
        np.testing.assert_array_equal(orc.philox4x64_10(ctr, key), _ref.numpy_philox_block(ctr, key))


# --------------------------------------------------------------------------- leverage
@pytest.mark.parametrize("n,r", [(7, 3), (40, 5), (200, 25), (25, 25)])
def test_leverage_matches_svd_and_definition(orc, n, r):
    g = np.random.default_rng(n * 100 + r)
    A = g.standard_normal((n, r)) * np.exp(g.standard_normal(r))
    lev, rank = orc.leverage(A)
    assert rank == r
    np.testing.assert_allclose(lev, _ref.svd_leverage(A), rtol=1e-10, atol=1e-13)
    # Definition 3.4 and the facts stated after it: sum = r, 0 <= l <= 1
    assert abs(lev.sum() - r) < 1e-10 * r
    assert lev.min() >= -1e-15 and lev.max() <= 1 + 1e-12
    # invariant to column scaling and to orthogonal mixing of the columns
    Q, _ = np.linalg.qr(g.standard_normal((r, r)))
    lev2, _ = orc.leverage(A @ Q * 3.7)
    np.testing.assert_allclose(lev2, lev, rtol=1e-10, atol=1e-13)


def test_leverage_rank_deficient(orc):
    g = np.random.default_rng(3)
    B = g.standard_normal((30, 3))
    A = np.hstack([B, B[:, :1] * 2.0, np.zeros((30, 1))])  # rank 3 of 5 columns
    lev, rank = orc.leverage(A)
    assert rank == 3
    np.testing.assert_allclose(lev, _ref.svd_leverage(B), rtol=1e-10, atol=1e-13)
    assert abs(lev.sum() - 3) < 1e-10


def test_krp_leverage_bound_lemma_5_1(orc):
    """l_i(Z) <= prod_k l_{i_k}(A_k) (Lemma 5.1) by brute force on explicit Z; the
    bound sums to r^d, and is attained by the Kronecker product."""
    g = np.random.default_rng(5)
    r = 3
    mats = [g.standard_normal((n, r)) for n in (5, 6, 4)]
    Z = _ref.khatri_rao(mats)
    levZ = _ref.svd_leverage(Z)
    levs = [orc.leverage(A)[0] for A in mats]
    bound = _ref.product_probs(levs)
    assert np.all(levZ <= bound + 1e-12)
    assert abs(bound.sum() - r ** 3) < 1e-9
    # the Kronecker product of the factors has exactly the product leverage scores
    K = np.kron(np.kron(mats[2], mats[1]), mats[0])
    np.testing.assert_allclose(_ref.svd_leverage(K), bound, rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------- sampling
def _dists(orc, dims, r, seed, skew=0.0):
    g = np.random.default_rng(seed)
    out = []
    for n in dims:
        A = g.standard_normal((n, r))
        if skew:
            A[: max(1, n // 5)] *= skew  # a few heavy rows: concentrated leverage
        out.append(orc.ModeDist(orc.leverage(A)[0], r))
    return out


def test_cdf_fixed_point(orc):
    g = np.random.default_rng(7)
    lev = g.random(1000)
    lev[::17] = 0.0
    lev *= 5 / lev.sum()  # leverage scores of a rank-5 matrix sum to 5
    d = orc.ModeDist(lev, 5)
    q = np.array([int(np.rint(math.ldexp(x / 5, 62))) for x in lev], dtype=np.uint64)
    np.testing.assert_array_equal(d.q, q)
    np.testing.assert_array_equal(d.C, np.cumsum(q, dtype=np.uint64))
    assert d.T == int(q.astype(object).sum())
    assert d.maxq == int(q.max()) and d.nnzq == int((q > 0).sum())


def test_inverse_cdf_draw_exact(orc):
    d = _dists(orc, [300], 4, 11, skew=8.0)[0]
    g = np.random.default_rng(12)
    for u in list(g.integers(0, 2**64, size=2000, dtype=np.uint64)) + [0, 2**64 - 1]:
        assert orc.draw(d, int(u)) == _ref.draw_ref(d.C, d.T, int(u))
    # rows with q = 0 are never drawn
    lev = np.ones(50)
    lev[10:20] = 0
    d0 = orc.ModeDist(lev, 1)
    for u in g.integers(0, 2**64, size=3000, dtype=np.uint64):
        assert not 10 <= orc.draw(d0, int(u)) < 20


def test_rnd_skrp_draws_and_weights_exact(orc):
    """Every slot of RndSkrp (Alg. 2) re-derived from numpy's Philox + searchsorted."""
    dims, r, seed, it, k = [13, 9, 11], 3, 99, 4, 2
    ds = _dists(orc, dims, r, 21, skew=5.0)
    tau = 2.0 ** -6
    idet, pv, sdet, pdet = orc.det_skrp(ds, tau, 200)
    assert sdet > 0
    srnd = 200 - sdet
    irnd, wrnd, att = orc.rnd_skrp(ds, srnd, tau, pdet, seed, it, k)
    ps = [d.p for d in ds]
    pfull = _ref.product_probs(ps)
    tries = 0
    for j in range(srnd):
        for a in range(4096):
            ctr = [j, a, k | (1 << 32), it]
            out = _ref.numpy_philox_block(ctr, [seed, 0])
            ii = [_ref.draw_ref(ds[t].C, ds[t].T, out[t]) for t in range(3)]
            key = ii[0] + dims[0] * (ii[1] + dims[1] * ii[2])
            tries += 1
            if pfull[key] <= tau:
                break
        assert irnd[j] == key
        assert wrnd[j] == math.sqrt((1.0 - pdet) / (pfull[key] * srnd))
    assert att == tries


def test_det_skrp_brute_force(orc):
    """DetSkrp's pruned enumeration (Section 5.3) equals {i : p_i > tau} over all N."""
    for seed, dims, tau in [(1, [20, 15, 12], 2.0 ** -9), (2, [40, 30], 2.0 ** -8),
                            (3, [8, 7, 6, 5], 2.0 ** -10), (4, [30, 30, 30], 1.0)]:
        ds = _dists(orc, dims, 3, seed, skew=6.0)
        pfull = _ref.product_probs([d.p for d in ds])
        want = np.nonzero(pfull > tau)[0].astype(np.uint64)
        idet, pv, sdet, pdet = orc.det_skrp(ds, tau, 10 ** 6)
        np.testing.assert_array_equal(idet, want)
        np.testing.assert_array_equal(pv, pfull[want.astype(np.int64)])
        assert pdet == math.fsum(pfull[want.astype(np.int64)])


def test_det_threshold_is_strict(orc):
    ds = _dists(orc, [10, 10], 2, 8, skew=4.0)
    pfull = _ref.product_probs([d.p for d in ds])
    tau = float(np.sort(pfull)[-5])  # exactly one of the product values
    idet, _, sdet, _ = orc.det_skrp(ds, tau, 1000)
    assert sdet == int((pfull > tau).sum())
    assert tau not in set(pfull[idet.astype(np.int64)])


def test_det_top_s_selection(orc):
    ds = _dists(orc, [12, 10], 2, 9, skew=3.0)
    pfull = _ref.product_probs([d.p for d in ds])
    tau = 0.0
    s = 17
    idet, pv, sdet, pdet = orc.det_skrp(ds, tau, s)
    order = sorted(range(pfull.size), key=lambda i: (-pfull[i], i))[:s]
    assert sdet == s
    np.testing.assert_array_equal(idet, np.array(sorted(order), dtype=np.uint64))
    assert pdet == math.fsum(pfull[sorted(order)])


def test_det_cap(orc):
    ds = _dists(orc, [50, 50, 50], 2, 10)
    with pytest.raises(orc.OracleError) as e:
        orc.det_skrp(ds, 1e-12, 1 << 20, cap=1000)
    assert e.value.code == orc.ERR_DET_CAP


def test_reject_limit(orc):
    ds = _dists(orc, [3, 3], 1, 4)
    # tau below every p_i: every draw is deterministic, nothing can be accepted
    with pytest.raises(orc.OracleError) as e:
        orc.rnd_skrp(ds, 5, 1e-9, 0.0, 0, 0, 0, reject_cap=50)
    assert e.value.code == orc.ERR_REJECT_LIMIT


def test_combine_repeats_norm_identity(orc):
    """||Omega_bar x|| = ||Omega x|| after combining (Section 4.1), for random x."""
    dims, r = [16, 14, 12], 3
    ds = _dists(orc, dims, r, 31, skew=10.0)
    tau = 2.0 ** -7
    s = 300
    res = orc.skrp_lev(ds, s, tau, 5, 1, 0)
    idet, _, sdet, pdet = orc.det_skrp(ds, tau, s)
    irnd, wrnd, _ = orc.rnd_skrp(ds, s - sdet, tau, pdet, 5, 1, 0)
    assert res["sdet"] == sdet and res["pdet"] == pdet
    np.testing.assert_array_equal(res["idx"][:sdet], idet)
    assert np.all(res["wgt"][:sdet] == 1.0) and np.all(res["cnt"][:sdet] == 1)
    tail = res["idx"][sdet:]
    assert np.all(np.diff(tail.astype(np.int64)) > 0)
    assert res["cnt"][sdet:].sum() == s - sdet
    uniq, cnt = np.unique(irnd, return_counts=True)
    np.testing.assert_array_equal(tail, uniq)
    np.testing.assert_array_equal(res["cnt"][sdet:], cnt)
    assert res["sbar"] == sdet + uniq.size
    g = np.random.default_rng(0)
    N = int(np.prod(dims))
    for _ in range(5):
        x = g.standard_normal(N)
        full = math.fsum(list(x[idet.astype(np.int64)] ** 2) + list((wrnd * x[irnd.astype(np.int64)]) ** 2))
        comb = math.fsum((res["wgt"] * x[res["idx"].astype(np.int64)]) ** 2)
        assert abs(full - comb) <= 1e-12 * full


def test_sampling_distribution_lemma_5_3(orc):
    """Chi-square of random-only draws against prod_k p_k (Lemma 5.3)."""
    dims, r = [6, 5, 4], 2
    ds = _dists(orc, dims, r, 41, skew=3.0)
    s = 60000
    irnd, _, _ = orc.rnd_skrp(ds, s, 1.0, 0.0, 123, 0, 0)
    pfull = _ref.product_probs([d.p for d in ds])
    obs = np.bincount(irnd.astype(np.int64), minlength=pfull.size)
    exp = pfull * s
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    dof = pfull.size - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_rejection_distribution(orc):
    """Accepted hybrid draws follow p_i / (1 - p_det) on the complement of D."""
    dims, r = [8, 6], 2
    ds = _dists(orc, dims, r, 43, skew=6.0)
    tau = 2.0 ** -5
    idet, _, sdet, pdet = orc.det_skrp(ds, tau, 10 ** 6)
    assert sdet > 0
    s = 60000
    irnd, _, _ = orc.rnd_skrp(ds, s, tau, pdet, 7, 0, 1)
    pfull = _ref.product_probs([d.p for d in ds])
    mask = pfull <= tau
    obs = np.bincount(irnd.astype(np.int64), minlength=pfull.size)
    assert obs[~mask].sum() == 0
    exp = pfull[mask] / pfull[mask].sum() * s
    chi2 = float(((obs[mask] - exp) ** 2 / exp).sum())
    dof = int(mask.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)
    assert abs(pfull[mask].sum() - (1 - pdet)) < 1e-12


def test_unbiased_sketch_lemma_3_3(orc):
    """E||Omega x||^2 = ||x||^2 for the hybrid sketch with combined rows (Lemma 3.3,
    Eqs. 4.2-4.4).  A wrong weight (s in place of s_rnd, a missing sqrt(c), a dropped
    (1 - p_det)) moves the mean by far more than the tolerance."""
    dims, r = [10, 8], 2
    ds = _dists(orc, dims, r, 47, skew=8.0)
    tau = 2.0 ** -6
    s = 40
    g = np.random.default_rng(1)
    x = g.standard_normal(int(np.prod(dims)))
    vals = []
    for it in range(3000):
        res = orc.skrp_lev(ds, s, tau, 17, it, 0)
        vals.append(math.fsum((res["wgt"] * x[res["idx"].astype(np.int64)]) ** 2))
    assert res["sdet"] >= 5  # a sizeable deterministic block
    vals = np.array(vals)
    mean, sem = vals.mean(), vals.std() / math.sqrt(vals.size)
    assert abs(mean - x @ x) < 4 * sem + 1e-12


def test_exact_sum_matches_fsum(orc):
    g = np.random.default_rng(2)
    for n in (1, 7, 1000, 50000):
        x = np.exp(g.uniform(-700, 5, size=n)) * g.random(n)
        assert orc.exact_sum(x) == math.fsum(x)
    x = np.array([1.0, 2.0 ** -53, 2.0 ** -53])  # tie breaking beyond double precision
    assert orc.exact_sum(x) == math.fsum(x)
    x = np.array([5e-324] * 3 + [2.0 ** -1070])
    assert orc.exact_sum(x) == math.fsum(x)


# --------------------------------------------------------------------------- sizes
def test_bijection_against_printed_sizes(orc):
    """Eq. 2.2: the number of rows of Z for the Uber mode-1 subproblem is the product
    of the other mode sizes, printed as N = 46,977,120 in Section 6.2; the Amazon
    per-mode row counts of Fig. 6.2 are 3e12, 9e12, 9e12 to one digit."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    uber = gold["tensors"]["uber"]["dims"]
    assert math.prod(uber[1:]) == gold["uber_mode1_rows"]
    amazon = gold["tensors"]["amazon"]["dims"]
    for k, approx in enumerate(gold["amazon_mode_rows_approx"]):
        N = math.prod(n for m, n in enumerate(amazon) if m != k)
        assert float(f"{N:.0e}") == approx
    # the largest key of the Uber mode-1 problem is N - 1 and fits comfortably in 64 bits
    coo = synth.random_sparse_tensor(uber, 1, seed=0)
    idx = orc.Index(synth.Coo(tuple(uber), [np.array([n - 1], np.int32) for n in uber],
                              np.array([1.0])))
    keys, off, ik, val = idx.export(0)
    assert int(keys[0]) == gold["uber_mode1_rows"] - 1 and ik[0] == uber[0] - 1


# --------------------------------------------------------------------------- index
def test_index_fibres(orc):
    coo = synth.random_sparse_tensor((9, 7, 5, 4), 400, seed=3)
    idx = orc.Index(coo)
    X = coo.dense()
    for k in range(4):
        keys, off, ik, val = idx.export(k)
        U = _ref.unfold(X, k)
        cols = np.nonzero(np.any(U != 0, axis=0))[0]
        np.testing.assert_array_equal(keys, cols.astype(np.uint64))
        for f, key in enumerate(keys):
            rows = ik[off[f]:off[f + 1]]
            assert np.all(np.diff(rows) > 0)
            np.testing.assert_array_equal(rows, np.nonzero(U[:, key])[0])
            np.testing.assert_array_equal(val[off[f]:off[f + 1]], U[rows, key])


def test_index_rejects_bad_coo(orc):
    coo = synth.random_sparse_tensor((5, 4, 3), 20, seed=1)
    bad = synth.Coo(coo.dims, [c.copy() for c in coo.idx], coo.vals)
    bad.idx[1][3] = 4
    with pytest.raises(orc.OracleError) as e:
        orc.Index(bad)
    assert e.value.code == orc.ERR_COO_RANGE
    dup = synth.Coo(coo.dims, [np.append(c, c[0]) for c in coo.idx], np.append(coo.vals, 1.0))
    with pytest.raises(orc.OracleError) as e:
        orc.Index(dup)
    assert e.value.code == orc.ERR_COO_DUP


# --------------------------------------------------------------------------- products
def _tiny_problem(seed=0, dims=(7, 6, 5), r=3, nnz=120):
    coo = synth.random_sparse_tensor(dims, nnz, seed=seed)
    facs = synth.gaussian_factors(dims, r, seed=seed + 1)
    return coo, facs


def test_sampled_mttkrp_all_rows_equals_dense(orc):
    """tau = 0 with s >= N takes every row once with weight 1, so the sampled MTTKRP
    and Gram equal X_(k) Z and Z^T Z (Eq. 1.1 via normal equations)."""
    coo, facs = _tiny_problem(dims=(7, 6, 5, 3), nnz=200)
    idx = orc.Index(coo)
    X = coo.dense()
    r = facs[0].shape[1]
    for k in range(4):
        others = [m for m in range(4) if m != k]
        ds = [orc.ModeDist(orc.leverage(facs[m])[0], r) for m in others]
        N = int(np.prod([coo.dims[m] for m in others]))
        res = orc.skrp_lev(ds, N, 0.0, 0, 0, k)
        assert res["sdet"] == N and res["sbar"] == N
        np.testing.assert_array_equal(res["idx"], np.arange(N, dtype=np.uint64))
        M, G, nz = orc.sampled_mttkrp(idx, k, facs, res["idx"], res["wgt"])
        Mref, Z = _ref.dense_mttkrp(X, facs, k)
        np.testing.assert_allclose(M, Mref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(G, Z.T @ Z, rtol=1e-12, atol=1e-12)
        assert nz == coo.nnz
        Me, Ge = orc.exact_mttkrp(idx, k, facs)
        np.testing.assert_allclose(Me, Mref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Ge, Z.T @ Z, rtol=1e-12, atol=1e-12)


def test_sampled_mttkrp_weights_and_empty_fibres(orc):
    coo, facs = _tiny_problem(dims=(6, 5, 4), nnz=30, seed=4)
    idx = orc.Index(coo)
    X = coo.dense()
    k = 0
    g = np.random.default_rng(0)
    keys = np.unique(g.integers(0, 20, size=12)).astype(np.uint64)
    w = g.uniform(0.5, 2.0, size=keys.size)
    M, G, nz = orc.sampled_mttkrp(idx, k, facs, keys, w)
    U = _ref.unfold(X, k)
    Z = _ref.khatri_rao([facs[1], facs[2]])
    Zs = Z[keys.astype(np.int64)] * w[:, None]
    Xs = U[:, keys.astype(np.int64)] * w[None, :]
    np.testing.assert_allclose(M, Xs @ Zs, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G, Zs.T @ Zs, rtol=1e-12, atol=1e-13)
    assert nz == int(np.count_nonzero(U[:, keys.astype(np.int64)]))


def test_solve_and_singular_fallback(orc):
    g = np.random.default_rng(5)
    B = g.standard_normal((40, 6))
    G = B.T @ B
    M = g.standard_normal((9, 6))
    A, rc = orc.solve(G, M)
    assert rc == 0
    np.testing.assert_allclose(A, np.linalg.solve(G, M.T).T, rtol=1e-11, atol=1e-12)
    Gs = G.copy()
    Gs[:, 5] = 0
    Gs[5, :] = 0
    A2, rc2 = orc.solve(Gs, M)
    assert rc2 == orc.WARN_SINGULAR_GRAM
    np.testing.assert_allclose(A2, M @ np.linalg.pinv(Gs), rtol=1e-9, atol=1e-11)


def test_normalize(orc):
    g = np.random.default_rng(6)
    A = g.standard_normal((20, 4))
    A[:, 2] = 0
    An, lam = orc.normalize(A)
    np.testing.assert_allclose(lam, np.linalg.norm(A, axis=0), rtol=1e-14)
    np.testing.assert_allclose(An[:, [0, 1, 3]], A[:, [0, 1, 3]] / lam[[0, 1, 3]], rtol=1e-14)
    assert np.all(An[:, 2] == 0)


def test_fit_matches_dense(orc):
    coo, facs = _tiny_problem(dims=(5, 4, 6), nnz=60, seed=7)
    idx = orc.Index(coo)
    lam = np.array([1.5, 0.3, 2.0])
    f = orc.fit(idx, facs, lam)
    X = coo.dense()
    Mdense = _ref.cp_dense(lam, facs)
    want = 1 - np.linalg.norm(X - Mdense) / np.linalg.norm(X)
    assert abs(f - want) < 1e-12


# --------------------------------------------------------------------------- updates
def test_mode_update_all_rows_is_cp_als_update(orc):
    """With tau = 0 and s >= N the randomized update is the CP-ALS update: A_k solves
    min ||Z B^T - X_(k)^T|| exactly (Eq. 1.1), here checked with numpy lstsq."""
    coo, facs = _tiny_problem(dims=(6, 5, 4), nnz=80, seed=8)
    idx = orc.Index(coo)
    X = coo.dense()
    r = 3
    for k in range(3):
        N = int(np.prod([n for m, n in enumerate(coo.dims) if m != k]))
        res = orc.mode_update(idx, facs, k, rank=r, samples=N, tau=0.0)
        _, Z = _ref.dense_mttkrp(X, facs, k)
        B = np.linalg.lstsq(Z, _ref.unfold(X, k).T, rcond=None)[0].T
        np.testing.assert_allclose(res["A"] * res["lam"], B, rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(np.linalg.norm(res["A"], axis=0), 1.0, rtol=1e-13)


def test_planted_exact_lowrank_fit_to_one(orc):
    """On an exactly rank-r tensor, both CP-ALS and CP-ARLS-LEV reach fit -> 1.  The fit
    of Eq. 5.1 evaluated as ||X||^2 - 2<X,M> + ||M||^2 cancels, so its floor is about
    sqrt(2^-52) = 1.5e-8 below 1; the check allows 1e-7."""
    coo, lam0, facs0 = synth.exact_lowrank_tensor((12, 10, 9), 3, seed=2, density=0.6)
    idx = orc.Index(coo)
    init = synth.gaussian_factors(coo.dims, 3, seed=1)
    _, _, f_als, _ = orc.cp_als(idx, init, rank=3, iters=200)
    assert f_als > 1 - 1e-7
    lam, fs, f, done, warn = orc.cp_arls_lev(idx, init, rank=3, samples=300, tau=1.0, iters=200,
                                             seed=3)
    assert f > 1 - 1e-7
    X = coo.dense()
    np.testing.assert_allclose(_ref.cp_dense(lam, fs), X, atol=1e-6 * np.abs(X).max())


def test_small_planted_close_to_cp_als(orc):
    """The 60x50x40 planted count tensor: CP-ARLS-LEV (random, s = 1024, 10 iters) lands
    near CP-ALS from the same start (the paper reports nearly equal fits, Section 6)."""
    coo = synth.small_planted_tensor(0)
    idx = orc.Index(coo)
    init = synth.gaussian_factors(coo.dims, 4, seed=0)
    _, _, f_als, _ = orc.cp_als(idx, init, rank=4, iters=10)
    _, _, f, _, _ = orc.cp_arls_lev(idx, init, rank=4, samples=1024, tau=1.0, iters=10, seed=0)
    assert 0.3 < f_als < 1
    assert abs(f - f_als) < 0.05


@pytest.mark.slow
def test_theorem_5_2_bound_holds(orc):
    """Theorem 5.2: with s = r^d max(C log(r/delta), 1/(delta eps)) samples drawn from
    the product leverage distribution, the sketched residual is within (1 + eps) of
    the optimum with probability at least 1 - delta."""
    dims, r = (12, 10, 8), 2
    g = np.random.default_rng(0)
    X = g.random(dims)
    coo = synth.Coo(dims, [c.astype(np.int32) for c in np.nonzero(X)], X[np.nonzero(X)])
    idx = orc.Index(coo)
    facs = synth.gaussian_factors(dims, r, seed=4)
    k, d = 2, 2
    delta, eps = 0.2, 0.5
    Cc = 144 / (1 - 1 / math.sqrt(2)) ** 2
    s = int(math.ceil(r ** d * max(Cc * math.log(r / delta), 1 / (delta * eps))))
    _, Z = _ref.dense_mttkrp(X, facs, k)
    Y = _ref.unfold(X, k).T
    Bopt = np.linalg.lstsq(Z, Y, rcond=None)[0]
    ropt = np.linalg.norm(Z @ Bopt - Y) ** 2
    ok = 0
    trials = 60
    for t in range(trials):
        res = orc.mode_update(idx, facs, k, rank=r, samples=s, tau=1.0, seed=t, it=t)
        B = (res["A"] * res["lam"]).T
        ok += np.linalg.norm(Z @ B - Y) ** 2 <= (1 + eps) * ropt
    assert ok >= (1 - delta) * trials


# --------------------------------------------------------------------------- estimated fit (Section 5.4)
def _brute_F(coo, factors, lam):
    """||X - M||^2 summed over every cell of the dense tensor."""
    M = np.zeros(coo.dims)
    for j in range(lam.shape[0]):
        T = lam[j]
        for A in factors:
            T = np.multiply.outer(T, A[:, j])
        M += T
    return float(((coo.dense() - M) ** 2).sum())


def test_fit_sample_draws_follow_their_definition(orc):
    """Every draw recomputed from numpy's Philox: nonzero slot j takes the nonzero at
    floor(u nnz / 2^64) in ascending linear-index order (np.lexsort, last mode most
    significant); zero slot j takes the first attempt whose uniform coordinates
    (floor(u_m n_m / 2^64)) miss every nonzero."""
    coo = synth.random_sparse_tensor((5, 7, 3, 4), 150, seed=4)
    X = orc.Index(coo)
    s_fit, alpha, seed = 301, 0.3, 77
    fs = orc.fit_sample(X, s_fit, alpha=alpha, seed=seed)
    cells = math.prod(coo.dims)
    s_nz = math.ceil(alpha * s_fit)
    assert (fs.s_nz, fs.s_z) == (s_nz, s_fit - s_nz)
    assert fs.phi[0] == coo.nnz / s_nz and fs.phi[1] == (cells - coo.nnz) / (s_fit - s_nz)
    order = np.lexsort(tuple(coo.idx))
    nz_set = set(zip(*(i.tolist() for i in coo.idx)))
    for j in range(s_nz):
        u = int(_ref.numpy_philox_block([j, 0, 2 << 32, 0], [seed, 0])[0])
        e = order[(u * coo.nnz) >> 64]
        assert tuple(int(c) for c in fs.coords[:, j]) == tuple(int(i[e]) for i in coo.idx)
        assert fs.xs[j] == coo.vals[e]
    attempts = 0
    for j in range(s_fit - s_nz):
        for a in range(4096):
            c = []
            for m, n in enumerate(coo.dims):
                u = int(_ref.numpy_philox_block([j, a, (2 << 32) | 1 | ((m // 4) << 16), 0], [seed, 0])[m % 4])
                c.append((u * n) >> 64)
            attempts += 1
            if tuple(c) not in nz_set:
                break
        assert tuple(int(x) for x in fs.coords[:, s_nz + j]) == tuple(c)
        assert fs.xs[s_nz + j] == 0.0
    assert fs.attempts == attempts


def test_fit_sample_strata_are_uniform(orc):
    """Chi-square: nonzero draws uniform over the nonzeros, zero draws uniform over
    the zero cells and never on a nonzero."""
    from scipy import stats
    coo = synth.random_sparse_tensor((4, 3, 2), 7, seed=2)
    X = orc.Index(coo)
    fs = orc.fit_sample(X, 40000, alpha=0.5, seed=5)
    lin = lambda c: c[0] + 4 * (c[1] + 3 * c[2])  # noqa: E731
    nz = {lin(c): e for e, c in enumerate(zip(*(i.tolist() for i in coo.idx)))}
    cnt_nz = np.zeros(coo.nnz)
    for j in range(fs.s_nz):
        e = nz[lin(fs.coords[:, j].tolist())]
        cnt_nz[e] += 1
        assert fs.xs[j] == coo.vals[e]
    zeros = [c for c in range(24) if c not in nz]
    cnt_z = np.zeros(24)
    for j in range(fs.s_nz, fs.s_nz + fs.s_z):
        cnt_z[lin(fs.coords[:, j].tolist())] += 1
    assert cnt_z[list(nz)].sum() == 0
    assert stats.chisquare(cnt_nz).pvalue > 1e-4
    assert stats.chisquare(cnt_z[zeros]).pvalue > 1e-4


def test_fit_estimate_exact_lowrank_is_one(orc):
    """A sparse tensor that is exactly its CP model: every sampled residual is zero
    (up to rounding) in both strata, so the estimated fit is 1."""
    coo, lam, facs = synth.exact_lowrank_tensor((9, 8, 7), 3, seed=1, density=0.4)
    X = orc.Index(coo)
    fs = orc.fit_sample(X, 5000, alpha=0.5, seed=3)
    assert fs.s_z > 0 and fs.s_nz > 0
    fit, F = orc.fit_estimate(X, fs, facs, lam)
    assert F <= 1e-24 * float((coo.vals ** 2).sum()) and fit > 1 - 1e-12
    # a model with one factor's rows permuted is far from X in both strata
    bad = [facs[0], facs[1][::-1].copy(), facs[2]]
    fit_bad, _ = orc.fit_estimate(X, fs, bad, lam)
    assert fit_bad < 0.9


def test_fit_estimate_is_unbiased(orc):
    """E[F_hat] = ||X - M||^2 (Section 5.4's weights make each stratum's sum
    unbiased): the mean over 400 independent samples is within 5 standard errors of
    the brute-force value, and the estimate with the zero-stratum weight
    prod(n) / s_z (instead of (prod(n) - nnz) / s_z) is not."""
    coo = synth.random_sparse_tensor((6, 5, 4), 40, seed=9)
    X = orc.Index(coo)
    g = np.random.default_rng(0)
    facs = [g.uniform(0.0, 1.0, size=(n, 2)) for n in coo.dims]
    lam = np.array([1.0, 0.5])
    F_true = _brute_F(coo, facs, lam)
    Fs, Fs_wrong = [], []
    cells = math.prod(coo.dims)
    for seed in range(400):
        fs = orc.fit_sample(X, 64, alpha=0.5, seed=seed)
        Fs.append(orc.fit_estimate(X, fs, facs, lam)[1])
        fs.phi = np.array([fs.phi[0], cells / fs.s_z])
        Fs_wrong.append(orc.fit_estimate(X, fs, facs, lam)[1])
    Fs, Fs_wrong = np.array(Fs), np.array(Fs_wrong)
    se = Fs.std(ddof=1) / math.sqrt(Fs.size)
    assert abs(Fs.mean() - F_true) < 5 * se
    assert abs(Fs_wrong.mean() - F_true) > 5 * se


def test_fit_sample_edge_cases(orc):
    # a tensor with no zero cell: the zero stratum is empty and the estimate exact
    # in expectation from the nonzeros alone
    dims = (3, 2, 2)
    full = np.stack(np.unravel_index(np.arange(12), dims, order="F"))
    coo = synth.Coo(dims, [c.astype(np.int32) for c in full], np.arange(1.0, 13.0))
    X = orc.Index(coo)
    fs = orc.fit_sample(X, 10, alpha=0.5, seed=1)
    assert (fs.s_nz, fs.s_z) == (5, 0) and fs.phi[1] == 0.0
    # alpha = 1: nonzeros only; alpha outside (0, 1] and s_fit < 1 are errors
    coo2 = synth.random_sparse_tensor((5, 4, 3), 10, seed=3)
    X2 = orc.Index(coo2)
    fs = orc.fit_sample(X2, 17, alpha=1.0, seed=2)
    assert (fs.s_nz, fs.s_z) == (17, 0)
    for bad in (dict(s_fit=0, alpha=0.5), dict(s_fit=8, alpha=0.0), dict(s_fit=8, alpha=1.5)):
        with pytest.raises(orc.OracleError):
            orc.fit_sample(X2, bad["s_fit"], alpha=bad["alpha"], seed=0)
    # a nearly full tensor with a rejection cap of 1 hits the limit
    coo3 = synth.random_sparse_tensor((4, 4, 4), 63, seed=1)
    with pytest.raises(orc.OracleError) as ei:
        orc.fit_sample(orc.Index(coo3), 200, alpha=0.5, seed=0, reject_cap=1)
    assert ei.value.code == orc.ERR_REJECT_LIMIT


# --------------------------------------------------------------------------- App. B distributions
def test_uniform_and_length_squared_scores(orc):
    """Uniform scores are r/n; length-squared scores are r times each row's share of
    ||A||_F^2; both sum to r, so p = score / r is a distribution.  The product of the
    length-squared factor distributions is the normalised bound of App. B,
    ||Z(i,:)||^2 <= prod_k ||A_k(i_k,:)||^2, checked on the explicit Khatri-Rao product."""
    g = np.random.default_rng(5)
    A = g.standard_normal((13, 4)) * np.array([1.0, 3.0, 0.2, 7.0])
    su, ru = orc.scores(A, orc.DIST_UNIFORM)
    assert ru == 4 and np.all(su == 4 / 13)
    sl, _ = orc.scores(A, orc.DIST_LENGTH_SQUARED)
    rows = np.linalg.norm(A, axis=1) ** 2
    np.testing.assert_allclose(sl, 4 * rows / np.linalg.norm(A) ** 2, rtol=1e-14)
    assert abs(sl.sum() - 4) < 1e-12
    mats = [g.standard_normal((n, 3)) for n in (5, 4, 6)]
    Z = _ref.khatri_rao(mats)
    bound = _ref.product_probs([np.linalg.norm(M, axis=1) ** 2 for M in mats])
    assert np.all((Z ** 2).sum(axis=1) <= bound * (1 + 1e-12))
    ps = [orc.scores(M, orc.DIST_LENGTH_SQUARED)[0] / 3 for M in mats]
    np.testing.assert_allclose(_ref.product_probs(ps), bound / bound.sum(), rtol=1e-12)


@pytest.mark.parametrize("dist", [1, 2])
def test_sampling_distribution_app_b(orc, dist):
    """Chi-square of random-only draws against the product of the per-factor uniform
    or length-squared distributions (the implicit product sampling of Lemma 5.3
    applies to any product distribution)."""
    g = np.random.default_rng(40 + dist)
    mats = [g.standard_normal((n, 2)) * np.exp(2 * g.standard_normal((n, 1))) for n in (6, 5, 4)]
    ds = [orc.ModeDist(orc.scores(M, dist)[0], 2) for M in mats]
    s = 60000
    irnd, _, _ = orc.rnd_skrp(ds, s, 1.0, 0.0, 321, 0, 0)
    pfull = _ref.product_probs([d.p for d in ds])
    if dist == 1:
        np.testing.assert_allclose(pfull, 1.0 / pfull.size, rtol=1e-12)
    obs = np.bincount(irnd.astype(np.int64), minlength=pfull.size)
    exp = pfull * s
    keep = exp > 0
    chi2 = float(((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum())
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


@pytest.mark.parametrize("dist", [1, 2])
def test_unbiased_sketch_app_b(orc, dist):
    """Lemma 3.3's unbiasedness E||Omega x||^2 = ||x||^2 holds for any sampling
    distribution positive where x is nonzero: uniform and length-squared, hybrid."""
    g = np.random.default_rng(50 + dist)
    mats = [g.standard_normal((n, 2)) * np.exp(g.standard_normal((n, 1))) for n in (10, 8)]
    ds = [orc.ModeDist(orc.scores(M, dist)[0], 2) for M in mats]
    tau = 2.0 ** -6
    x = g.standard_normal(80)
    vals = []
    for it in range(3000):
        res = orc.skrp_lev(ds, 40, tau, 19, it, 0)
        vals.append(math.fsum((res["wgt"] * x[res["idx"].astype(np.int64)]) ** 2))
    vals = np.array(vals)
    mean, sem = vals.mean(), vals.std() / math.sqrt(vals.size)
    assert abs(mean - x @ x) < 4 * sem + 1e-12


def test_app_b_all_rows_is_cp_als(orc):
    """With tau = 0 every row of positive probability is deterministic (weight 1), so
    an update under any of the three distributions is the exact CP-ALS update when
    all probabilities are positive."""
    coo = synth.random_sparse_tensor((6, 5, 4), 60, seed=8)
    X = orc.Index(coo)
    facs = synth.gaussian_factors(coo.dims, 3, seed=9)
    outs = [orc.mode_update(X, facs, 1, rank=3, samples=24, tau=0.0, distribution=dist) for dist in (0, 1, 2)]
    M, G = orc.exact_mttkrp(X, 1, facs)
    A, _ = orc.solve(G, M)
    An, _ = orc.normalize(A)
    for o in outs:
        assert o["sdet"] == 24
        np.testing.assert_allclose(o["A"], An, rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------------------- RRF initialisation (App. F)
def test_rrf_init_is_sampled_unfolding_times_omega(orc):
    """A = X_(k)(:, S) Omega from the dense mode-k unfolding (columns ordered by the
    linear key of Eq. 2.2 over the other modes, first fastest), S recomputed from
    numpy's Philox over the nonzero columns; every mode of a 4-way tensor."""
    coo = synth.random_sparse_tensor((5, 7, 3, 4), 90, seed=6)
    X = orc.Index(coo)
    Xd = coo.dense()
    g = np.random.default_rng(2)
    s_init, r, seed = 37, 3, 11
    for k in range(4):
        # columns of the unfolding: key = sum_t i_t prod_{u<t} n_u, first other mode fastest
        Xk = np.moveaxis(Xd, k, 0).reshape(coo.dims[k], -1, order="F")
        nzcols = np.nonzero(np.abs(Xk).sum(axis=0))[0]
        assert nzcols.size == X.nfib(k)
        omega = g.standard_normal((s_init, r))
        cols = []
        for j in range(s_init):
            u = int(_ref.numpy_philox_block([j, 0, (3 << 32) | k, 0], [seed, 0])[0])
            cols.append(nzcols[(u * nzcols.size) >> 64])
        want = Xk[:, cols] @ omega
        got = orc.rrf_init(X, k, omega, seed=seed)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    with pytest.raises(orc.OracleError):
        orc.rrf_init(X, 0, np.zeros((0, 2)))  # s_init = 0
