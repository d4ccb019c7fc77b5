"""Reproducibility of the FP64 path and long-run parity with the FP64 oracle.

Every FP64 sum of the update is taken in a fixed order: the Grams and the fit add
their blocks' partial sums in block order, and the sampled MTTKRP (for tensors of up
to 2^24 nonzeros) sorts its items by row and adds each row's terms in sample order.
Two runs from the same inputs therefore give the same factors bit for bit, even
after many iterations whose samples depend on every bit of the previous factors,
and a batch of decompositions gives what the same calls give one at a time.
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


@pytest.mark.slow
def test_fp64_reruns_bit_identical_uber_shaped_50_iterations():
    """The 183x24x1140x1717 planted tensor (3.3M nonzeros), r = 25, s = 2^17,
    tau = 2^-17: two 50-iteration FP64 runs on separate indices agree bit for bit."""
    coo = synth.uber_like_tensor(0)
    init = synth.gaussian_factors(coo.dims, 25, seed=0)
    outs = []
    for _ in range(2):
        gi = cpa.cpa_index_build(coo)
        res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=25, samples=2 ** 17, tau=2.0 ** -17, iters=50,
                              seed=0)
        outs.append(([f.cpu().numpy() for f in res.factors], res.lam.cpu().numpy(), res.fit))
        gi.free()
    (fa, la, fita), (fb, lb, fitb) = outs
    for a, b in zip(fa, fb):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(la, lb)
    assert fita == fitb


def test_long_run_rows_bit_exact_against_oracle():
    """A 4-way planted count tensor with 2e5 nonzeros (planted rank 25, Zipf(1.1)),
    r = 25, s = 2^14, hybrid sampling: 10 outer iterations of single mode updates, the
    GPU and the oracle each continuing from its own factors.  At every update:
    * the sampled rows, counts and sample sizes are equal bit for bit (the oracle on its
      own trajectory);
    * the GPU's new factor and lambda are within 1e-10 of the oracle's update taken from
      the GPU's current factors (each step's arithmetic, at every step of the run).
    The two trajectories' factors are held to 1e-10 for the first five iterations only:
    the early iterations of Alg. 3 from a random start amplify any difference in the last
    bits (the oracle itself, started from factors perturbed by 1e-15 relative, ends about
    1e-10 away from its unperturbed run after 10 iterations)."""
    dims, r, s = (120, 90, 110, 80), 25, 2 ** 14
    coo = synth.planted_cp_tensor(dims, r, target_nnz=200000, seed=31, zipf_alpha=1.1)
    assert coo.nnz >= 196000
    init = synth.gaussian_factors(dims, r, seed=32)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    fg = [cu(a) for a in init]
    fo = [a.copy() for a in init]
    for it in range(10):
        for k in range(len(dims)):
            before = [f.cpu().numpy() for f in fg]
            got = cpa.cpa_mode_update(gi, fg, k, rank=r, samples=s, tau=1.0 / s, seed=5, it=it)
            ref = oracle.mode_update(oi, fo, k, rank=r, samples=s, tau=1.0 / s, seed=5, it=it)
            one = oracle.mode_update(oi, before, k, rank=r, samples=s, tau=1.0 / s, seed=5, it=it)
            assert got["sbar"] == ref["sbar"] and got["sdet"] == ref["sdet"], (it, k)
            np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), ref["idx"])
            np.testing.assert_array_equal(got["cnt"].cpu().numpy().astype(np.uint32), ref["cnt"])
            np.testing.assert_array_equal(got["idx"].cpu().numpy().astype(np.uint64), one["idx"])
            fo[k] = ref["A"]
            step = relerr(fg[k].cpu().numpy(), one["A"])
            assert step < 1e-10, (it, k, step)
            assert relerr(got["lam"].cpu().numpy(), one["lam"]) < 1e-10, (it, k)
            if it < 5:
                e = relerr(fg[k].cpu().numpy(), ref["A"])
                assert e < 1e-10, (it, k, e)


@pytest.mark.parametrize("dims,nnz,k", [((2, 300, 200), 60000, 0), ((5, 70, 90), 25000, 0),
                                        ((40, 30, 20), 8000, 2)])
def test_sampled_mttkrp_rows_across_tiles(dims, nnz, k):
    """Rows whose sampled nonzeros span many 128-item tiles (two or five rows in mode
    0) and rows inside one tile: M equals the oracle's within 1e-12, and two calls
    give the same M bit for bit."""
    coo = synth.random_sparse_tensor(dims, nnz, seed=41)
    r = 7
    facs = synth.gaussian_factors(dims, r, seed=42)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    others = [m for m in range(3) if m != k]
    ds = [oracle.ModeDist(oracle.leverage(facs[m])[0], r) for m in others]
    s = 4000
    smp = oracle.skrp_lev(ds, s, 1.0 / s, 3, 0, k)
    Mr, Gr, nz = oracle.sampled_mttkrp(oi, k, facs, smp["idx"], smp["wgt"])
    outs = []
    for _ in range(2):
        M, G, nzg = cpa.cpa_sampled_mttkrp(gi, k, [cu(a) for a in facs], cu(smp["idx"]), cu(smp["wgt"]))
        outs.append(M.cpu().numpy())
        assert nzg == nz
        assert relerr(G.cpu().numpy(), Gr) < 1e-12
    assert relerr(outs[0], Mr) < 1e-12
    np.testing.assert_array_equal(outs[0], outs[1])


def test_batched_fp64_equals_single_calls_bit_for_bit():
    """Batched decompositions in FP64 give the single calls' factors and fits bit for
    bit, whatever SM budget the batch's kernels were sized for."""
    shapes = [((40, 30, 20), 3000, 4, 128, 1.0 / 128), ((25, 18, 30, 12), 6000, 7, 1024, 1.0 / 1024),
              ((90, 40, 33), 5000, 5, 256, 1.0 / 256)]
    probs = []
    for i, (d, nnz, r, s, tau) in enumerate(shapes):
        coo = synth.random_sparse_tensor(d, nnz, seed=50 + i)
        init = synth.gaussian_factors(d, r, seed=60 + i)
        probs.append(dict(index=cpa.cpa_index_build(coo), init=init, factors=[cu(a) for a in init], rank=r,
                          samples=s, tau=tau, iters=3, seed=i, precision=binding.FP64))
    batch = cpa.Batch(probs, autotune=1)
    batch.run()
    fits = batch.fits()
    for i, p in enumerate(probs):
        ref = cpa.cp_arls_lev(p["index"], [cu(a) for a in p["init"]], rank=p["rank"], samples=p["samples"],
                              tau=p["tau"], iters=p["iters"], seed=p["seed"])
        for m in range(len(ref.factors)):
            np.testing.assert_array_equal(p["factors"][m].cpu().numpy(), ref.factors[m].cpu().numpy())
        assert fits[i] == ref.fit
