"""Batched decompositions (one CUDA graph for many independent cp_arls_lev calls):
every problem's result equals the same call made on its own (same samples; the
sums differ only in the order of atomic additions), and a second run continues the
decompositions like a call with the iteration offset advanced."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_16438_gb300 as cpa  # noqa: E402
from paper_2006_16438_gb300 import binding  # noqa: E402

# s well below the number of Khatri-Rao rows of every mode (else the rejection loop
# of Alg. 2 can hit its cap, as it would in a single call)
SHAPES = [((40, 30, 20), 3000, 4, 128, 1.0 / 128), ((25, 18, 30, 12), 6000, 7, 1024, 1.0 / 1024),
          ((60, 50, 40), 4000, 10, 512, 1.0), ((90, 40, 33), 5000, 5, 256, 1.0 / 256)]


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _problems(precision=binding.FP64, iters=2):
    out = []
    for i, (dims, nnz, r, s, tau) in enumerate(SHAPES):
        coo = synth.random_sparse_tensor(dims, nnz, seed=10 + i)
        init = synth.gaussian_factors(dims, r, seed=20 + i)
        out.append(dict(index=cpa.cpa_index_build(coo), init=init, rank=r, samples=s, tau=tau, iters=iters,
                        seed=i, precision=precision))
    return out


@pytest.mark.parametrize("autotune", [0, 1])
def test_batch_matches_single_calls_and_continues(autotune):
    probs = _problems()
    for p in probs:
        p["factors"] = [torch.from_numpy(a).cuda() for a in p["init"]]
    batch = cpa.Batch(probs, autotune=autotune)
    refs = [[torch.from_numpy(a).cuda() for a in p["init"]] for p in probs]
    for run in range(2):
        batch.run()
        fits = batch.fits()
        for i, p in enumerate(probs):
            ref = cpa.cp_arls_lev(p["index"], refs[i], rank=p["rank"], samples=p["samples"], tau=p["tau"],
                                  iters=p["iters"], seed=p["seed"], iter_offset=run * p["iters"])
            for m in range(len(ref.factors)):
                assert relerr(p["factors"][m].cpu().numpy(), ref.factors[m].cpu().numpy()) < 1e-10
            assert relerr(batch.lams[i].cpu().numpy(), ref.lam.cpu().numpy()) < 1e-10
            assert abs(fits[i] - ref.fit) < 1e-10
            refs[i] = ref.factors
    info = batch.info()
    assert info["kernels"] > 0 and info["sm_budget"] > 0
    if autotune:
        assert all(b > 0 for b in info["candidates"]) and all(ms > 0 for ms in info["candidate_ms"])


def test_batch_rejects_fit_stopping_rule():
    probs = _problems(iters=1)[:1]
    probs[0]["factors"] = [torch.from_numpy(a).cuda() for a in probs[0]["init"]]
    probs[0]["tau"] = 1.0 / (4 * probs[0]["samples"])  # tau * s < 1: host top-s step
    with pytest.raises(binding.CpaError):
        cpa.Batch(probs, autotune=0)
