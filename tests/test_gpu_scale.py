"""The 4,821,207 x 1,774,269 x 1,805,187 configuration (int32 COO, FP32 count values,
Zipf(1.1) popularity, rank 25, s = 2^17, tau = 2^-17, mixed precision), generated on
the GPU.  The default run takes 1/16 of its 1.74e9 nonzeros (the shape is kept);
CPA_SCALE_FRACTION=1 runs the full size.

Checked at that size (the oracle's own index would not fit a test): one mixed-
precision mode update runs; for the rows it sampled, the FP64 sampled MTTKRP and
sampled Gram of the library equal their definitions (Sec. 5.3:
M(i, :) = sum_j w_j^2 x(i, key_j) z_j and G = sum_j w_j^2 z_j z_j^T) recomputed row by
row from the COO; the leverage scores of every factor sum to the rank (Def. 3.4); one
outer iteration of cp_arls_lev in mixed precision gives a finite fit.
"""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_16438_gb300 as cpa  # noqa: E402
from paper_2006_16438_gb300 import binding  # noqa: E402
from synth import gpu as sgpu  # noqa: E402

DIMS = (4_821_207, 1_774_269, 1_805_187)
FULL_NNZ = 1_740_000_000
RANK, S, TAU = 25, 2 ** 17, 2.0 ** -17


@pytest.fixture(scope="module")
def scale_tensor():
    frac = float(os.environ.get("CPA_SCALE_FRACTION", 1.0 / 16))
    t0 = time.perf_counter()
    idx, vals = sgpu.planted_cp_tensor_gpu(DIMS, RANK, events=int(1.5 * FULL_NNZ * frac), seed=0,
                                           zipf_alpha=1.1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    index = cpa.cpa_index_build(DIMS, device_tensors=(idx, vals))
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    factors = [torch.randn(n, RANK, dtype=torch.float64, device="cuda", generator=g) for n in DIMS]
    print(f"\nscale tensor: nnz={vals.numel()}, generated in {t1 - t0:.1f} s, index built in {t2 - t1:.1f} s")
    return dict(idx=idx, vals=vals, index=index, factors=factors)


def test_sampled_products_equal_their_definition_at_scale(scale_tensor):
    idx, vals, index = scale_tensor["idx"], scale_tensor["vals"], scale_tensor["index"]
    orig = [f.clone() for f in scale_tensor["factors"]]
    fs = [f.clone() for f in orig]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = cpa.cpa_mode_update(index, fs, 0, rank=RANK, samples=S, tau=TAU, seed=0, it=0, precision=binding.MIXED)
    torch.cuda.synchronize()
    print(f"mixed-precision mode update at scale: {1e3 * (time.perf_counter() - t0):.1f} ms (incl. setup)")
    assert 0 < res["sbar"] <= S and torch.all(res["wgt"] > 0)
    keys, wgt = res["idx"], res["wgt"]
    M, G, nz = cpa.cpa_sampled_mttkrp(index, 0, orig, keys, wgt)
    # the KRP rows of the sampled keys (other modes 1, 2; mode 1 fastest, Eq. 2.2)
    k = keys.to(torch.int64)
    i1, i2 = k % DIMS[1], k // DIMS[1]
    z = orig[1][i1] * orig[2][i2]
    w2 = (wgt * wgt)[:, None]
    G_def = (w2 * z).T @ z
    assert float((G - G_def).abs().max() / G_def.abs().max()) < 1e-12
    # rows of M: the heaviest three and two others, each from the COO directly
    norms = M.norm(dim=1)
    rows = torch.cat([torch.topk(norms, 3).indices, torch.tensor([0, DIMS[0] // 2], device="cuda")])
    order = torch.argsort(k)
    ks = k[order]
    for i in rows.tolist():
        pos = torch.nonzero(idx[0] == i).flatten()
        lin = idx[1][pos].to(torch.int64) + DIMS[1] * idx[2][pos].to(torch.int64)
        at = torch.searchsorted(ks, lin).clamp_max(ks.numel() - 1)
        hit = ks[at] == lin
        j = order[at[hit]]
        x = vals[pos[hit]].to(torch.float64)[:, None]
        row = (w2[j] * x * z[j]).sum(dim=0)
        ref = float(row.abs().max())
        assert float((M[i] - row).abs().max()) <= 1e-10 * max(ref, 1e-300)


def test_leverage_sums_to_rank_and_iteration_runs_at_scale(scale_tensor):
    for f in scale_tensor["factors"]:
        lev, _ = cpa.cpa_leverage(f)
        assert abs(float(lev.sum()) - RANK) < 1e-8 * RANK
    fs = [f.clone() for f in scale_tensor["factors"]]
    out = cpa.cp_arls_lev(scale_tensor["index"], fs, rank=RANK, samples=S, tau=TAU, iters=1, seed=0,
                          precision=binding.MIXED)  # first call: workspace and graphs
    assert np.isfinite(out.fit)
    for fit_mode, what in ((binding.FIT_NONE, "no fit"), (binding.FIT_EXACT, "exact fit")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = cpa.cp_arls_lev(scale_tensor["index"], out.factors, rank=RANK, samples=S, tau=TAU, iters=2, seed=0,
                              iter_offset=1, precision=binding.MIXED, fit_mode=fit_mode)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"2 outer iterations (6 mode updates) + {what}, mixed precision: {1e3 * dt:.1f} ms "
              f"({6 / dt:.1f} mode updates/s), fit {out.fit:.4f}")
    assert np.isfinite(out.fit)
