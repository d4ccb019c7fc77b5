"""Parity of the estimated fit (Section 5.4) on the GPU with the FP64 CPU oracle,
through the C ABI.

The element sample is integer work decided by Philox words and index probes, so
coordinates, values, counts, weights and the number of zero-cell attempts must
match bit for bit.  The FP64 estimate F_hat must match within 1e-12 relative (the
two sides sum the same terms in different orders), the fit within 1e-10; in mixed
precision (FP32 model values) the fit within 1e-4, the tolerance of the mixed path.
"""
import math

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


def _factors(dims, r, seed):
    g = np.random.default_rng(seed)
    return [g.standard_normal((n, r)) for n in dims], g.uniform(0.5, 2.0, size=r)


def _check_sample(gs, os_):
    assert (gs.s_nz, gs.s_z, gs.attempts) == (os_.s_nz, os_.s_z, os_.attempts)
    assert gs.phi == tuple(os_.phi)
    np.testing.assert_array_equal(gs.coords.cpu().numpy(), os_.coords)
    np.testing.assert_array_equal(gs.xs.cpu().numpy(), os_.xs)


CASES = [
    # (name, tensor, s_fit, alpha, seed)
    ("small-3way", lambda: synth.small_planted_tensor(0), 5000, 0.5, 1),
    ("ragged-4way", lambda: synth.random_sparse_tensor((13, 7, 29, 5), 3001, seed=2), 12345, 0.3, 7),
    ("dense-ish", lambda: synth.random_sparse_tensor((9, 8, 7), 400, seed=3), 20011, 0.5, 2),
    ("f32-values", lambda: synth.random_sparse_tensor((31, 17, 23), 2500, seed=4).as_dtype(np.float32), 7777,
     0.6, 3),
]


@pytest.mark.parametrize("name,make,s_fit,alpha,seed", CASES, ids=[c[0] for c in CASES])
def test_fit_sample_and_estimate_match_oracle(name, make, s_fit, alpha, seed):
    coo = make()
    X = cpa.cpa_index_build(coo, dtype=coo.vals.dtype)
    Xo = oracle.Index(coo.as_dtype(np.float64))
    gs = cpa.cpa_fit_sample(X, s_fit, alpha=alpha, seed=seed)
    os_ = oracle.fit_sample(Xo, s_fit, alpha=alpha, seed=seed)
    _check_sample(gs, os_)
    facs, lam = _factors(coo.dims, 6, seed)
    fit_o, F_o = oracle.fit_estimate(Xo, os_, facs, lam)
    fit_g, F_g = cpa.cpa_fit_estimate(X, gs, [torch.from_numpy(f) for f in facs], torch.from_numpy(lam))
    assert abs(F_g - F_o) <= 1e-12 * F_o
    assert abs(fit_g - fit_o) <= 1e-10
    fit_m, _ = cpa.cpa_fit_estimate(X, gs, [torch.from_numpy(f) for f in facs], torch.from_numpy(lam),
                                    precision=binding.MIXED)
    assert abs(fit_m - fit_o) <= 1e-4


@pytest.mark.parametrize("r", [1, 8, 9, 16, 25, 33, 64])
def test_estimate_all_rank_widths(r):
    coo = synth.random_sparse_tensor((40, 30, 20), 3000, seed=r)
    X = cpa.cpa_index_build(coo)
    Xo = oracle.Index(coo)
    gs = cpa.cpa_fit_sample(X, 3333, seed=r)
    os_ = oracle.fit_sample(Xo, 3333, seed=r)
    _check_sample(gs, os_)
    facs, lam = _factors(coo.dims, r, 100 + r)
    fit_o, F_o = oracle.fit_estimate(Xo, os_, facs, lam)
    fit_g, F_g = cpa.cpa_fit_estimate(X, gs, [torch.from_numpy(f) for f in facs], torch.from_numpy(lam))
    assert abs(F_g - F_o) <= 1e-12 * F_o


def test_uber_shape_sample_bit_exact():
    """The 183 x 24 x 1140 x 1717 planted tensor (3.3M nonzeros), 2^20 samples: the
    directory/hash probes of the zero rejections and the position search of the
    nonzero draws over the full index."""
    coo = synth.uber_like_tensor(0)
    X = cpa.cpa_index_build(coo)
    Xo = oracle.Index(coo)
    gs = cpa.cpa_fit_sample(X, 1 << 20, seed=5)
    os_ = oracle.fit_sample(Xo, 1 << 20, seed=5)
    _check_sample(gs, os_)


def test_edge_cases():
    # no zero cell: the zero stratum is empty
    dims = (3, 2, 2)
    full = np.stack(np.unravel_index(np.arange(12), dims, order="F"))
    coo = synth.Coo(dims, [c.astype(np.int32) for c in full], np.arange(1.0, 13.0))
    X = cpa.cpa_index_build(coo)
    gs = cpa.cpa_fit_sample(X, 10, seed=1)
    assert (gs.s_nz, gs.s_z) == (5, 0) and gs.phi[1] == 0.0
    _check_sample(gs, oracle.fit_sample(oracle.Index(coo), 10, seed=1))
    # one sample; alpha = 1
    coo2 = synth.random_sparse_tensor((5, 4, 3), 10, seed=3)
    X2 = cpa.cpa_index_build(coo2)
    for s_fit, alpha in ((1, 0.5), (17, 1.0), (2, 0.01)):
        _check_sample(cpa.cpa_fit_sample(X2, s_fit, alpha=alpha, seed=4),
                      oracle.fit_sample(oracle.Index(coo2), s_fit, alpha=alpha, seed=4))
    for s_fit, alpha in ((0, 0.5), (8, 0.0), (8, 1.5)):
        with pytest.raises(cpa.CpaError) as ei:
            cpa.cpa_fit_sample(X2, s_fit, alpha=alpha)
        assert ei.value.code == binding.ERR_ARG
    # a nearly full tensor with one draw allowed per zero slot: the rejection limit is
    # reported as a status (the kernel returns), and the device stays usable
    coo3 = synth.random_sparse_tensor((4, 4, 4), 63, seed=1)
    X3 = cpa.cpa_index_build(coo3)
    with pytest.raises(cpa.CpaError) as ei:
        cpa.cpa_fit_sample(X3, 200, seed=0, reject_cap=1)
    assert ei.value.code == binding.ERR_REJECT_LIMIT
    _check_sample(cpa.cpa_fit_sample(X3, 200, seed=0), oracle.fit_sample(oracle.Index(coo3), 200, seed=0))


@pytest.mark.parametrize("precision", [binding.FP64, binding.MIXED])
def test_cp_arls_lev_estimated_fit(precision):
    """The fit that cp_arls_lev reports with CPA_FIT_ESTIMATED is the oracle's
    estimate of the returned model on the oracle's sample (same seed and s_fit), and
    the stopping rule runs on it."""
    coo = synth.small_planted_tensor(0)
    X = cpa.cpa_index_build(coo)
    Xo = oracle.Index(coo)
    init = synth.gaussian_factors(coo.dims, 4, seed=0)
    s_fit = 1 << 14
    res = cpa.cp_arls_lev(X, [torch.from_numpy(a) for a in init], rank=4, samples=1024, tau=1.0, iters=10,
                          seed=3, fit_mode=binding.FIT_ESTIMATED, fit_samples=s_fit, fit_alpha=0.5,
                          precision=precision)
    os_ = oracle.fit_sample(Xo, s_fit, seed=3)
    fit_o, _ = oracle.fit_estimate(Xo, os_, [f.cpu().numpy() for f in res.factors], res.lam.cpu().numpy())
    tol = 1e-10 if precision == binding.FP64 else 1e-4
    assert abs(res.fit - fit_o) <= tol
    # the exact fit of the same model is close to the estimate
    exact = oracle.fit(Xo, [f.cpu().numpy() for f in res.factors], res.lam.cpu().numpy())
    assert abs(res.fit - exact) < 0.05
    # a second call reuses the sample (same options); the stopping rule on the estimate
    res2 = cpa.cp_arls_lev(X, res.factors, rank=4, samples=1024, tau=1.0, iters=200, seed=3, tol=1e-4,
                           patience=3, fit_mode=binding.FIT_ESTIMATED, fit_samples=s_fit, precision=precision)
    assert res2.stats["epochs"] >= 3 and np.isfinite(res2.fit)
    assert res2.stats["iters_done"] == 5 * res2.stats["epochs"] or res2.stats["iters_done"] == 200


def test_batch_with_estimated_fit():
    coo = synth.small_planted_tensor(1)
    X = cpa.cpa_index_build(coo)
    Xo = oracle.Index(coo)
    probs = [dict(index=X, factors=[torch.from_numpy(a).cuda() for a in synth.gaussian_factors(coo.dims, 4, seed=s)],
                  rank=4, samples=1024, tau=1.0, iters=5, seed=s, fit_mode=binding.FIT_ESTIMATED,
                  fit_samples=4096)
             for s in range(3)]
    b = cpa.Batch(probs, autotune=False)
    b.run()
    for i, p in enumerate(probs):
        os_ = oracle.fit_sample(Xo, 4096, seed=p["seed"])
        fit_o, _ = oracle.fit_estimate(Xo, os_, [f.cpu().numpy() for f in b.factors[i]], b.lams[i].cpu().numpy())
        assert abs(b.fits()[i] - fit_o) <= 1e-10
    b.free()


def test_estimate_at_uber_shape_equals_definition():
    """2^22 samples of the Uber-shaped tensor and a fitted model: the kernel's F_hat
    equals its definition recomputed with torch over the same sample, and is of the
    size of the exact residual (printed beside the exact fit)."""
    coo = synth.uber_like_tensor(0)
    X = cpa.cpa_index_build(coo)
    init = synth.gaussian_factors(coo.dims, 25, seed=0)
    res = cpa.cp_arls_lev(X, [torch.from_numpy(a) for a in init], rank=25, samples=1 << 17, tau=2.0 ** -17,
                          iters=10, seed=0, fit_mode=binding.FIT_EXACT)
    gs = cpa.cpa_fit_sample(X, 1 << 22, seed=0)
    est, F = cpa.cpa_fit_estimate(X, gs, res.factors, res.lam)
    v = res.lam[None, :].expand(gs.xs.numel(), -1).clone()
    for m, A in enumerate(res.factors):
        v *= A[gs.coords[m].to(torch.int64)]
    mv = v.sum(dim=1)
    phi = torch.full((mv.numel(),), gs.phi[1], dtype=torch.float64, device="cuda")
    phi[:gs.s_nz] = gs.phi[0]
    F_def = float((phi * (mv - gs.xs) ** 2).sum())
    # rounding of each model value scales with sum_c |lambda_c prod A|, and the
    # residuals of a fitted model cancel: bound the difference by those magnitudes
    scale = float((phi * (gs.xs ** 2 + v.abs().sum(dim=1) ** 2)).sum())
    assert abs(F - F_def) <= 1e-12 * scale
    print(f"uber-shape: exact fit {res.fit:.5f}, estimated (2^22 samples) {est:.5f}")
    assert abs(est - res.fit) < 0.05
