"""Mixed precision against the FP64 oracle at the stated tolerances, with the sampling
taken out of the comparison: tau = 0 and s at least the number of Khatri-Rao rows of
every mode make every row deterministic (each update is then the exact least-squares
update of CP-ALS), so the two runs differ only by FP32 arithmetic.  Factors and lambda
must agree within 2e-4 relative and the fit within 1e-4 absolute after 10 outer
iterations; the measured errors per result are printed."""
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


CASES = [
    ("planted 60x50x40, rank 4", lambda: synth.small_planted_tensor(0), 4, 3000),
    ("planted 40x30x20, rank 5, Zipf(1.1)",
     lambda: synth.planted_cp_tensor((40, 30, 20), 5, target_nnz=6000, seed=3, zipf_alpha=1.1), 5, 1200),
    ("planted 30x25x20x15, rank 6", lambda: synth.planted_cp_tensor((30, 25, 20, 15), 6, target_nnz=9000, seed=4),
     6, 15000),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mixed_whole_run_without_sampling_within_tolerance(case):
    name, make, r, s = CASES[case]
    coo = make()
    dims = coo.dims
    for k in range(len(dims)):
        assert s >= int(np.prod([n for m, n in enumerate(dims) if m != k]))
    init = synth.gaussian_factors(dims, r, seed=0)
    gi = cpa.cpa_index_build(coo)
    res = cpa.cp_arls_lev(gi, [torch.from_numpy(a).cuda() for a in init], rank=r, samples=s, tau=0.0, iters=10,
                          seed=0, precision=binding.MIXED)
    oi = oracle.Index(coo)
    lam, fs, fit, _, _ = oracle.cp_arls_lev(oi, init, rank=r, samples=s, tau=0.0, iters=10, seed=0)
    ef = [relerr(a.cpu().numpy(), b) for a, b in zip(res.factors, fs)]
    el = relerr(res.lam.cpu().numpy(), lam)
    efit = abs(res.fit - fit)
    print(f"{name}: factor rel err {['%.1e' % e for e in ef]}, lambda {el:.1e}, fit {efit:.1e}")
    assert max(ef) < 2e-4, ef
    assert el < 2e-4, el
    assert efit < 1e-4, efit
