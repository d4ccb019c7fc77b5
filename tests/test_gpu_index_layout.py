"""The fibre index built in segments and with narrow stored offsets (Section 5.3
index, the layout used for tensors of billions of nonzeros).

The builder splits the nonzeros of every mode into ranges of the top key field
(CPA_INDEX_SEGMENT_NNZ sets the largest segment) and stores fibre offsets as their low
bits plus the fibres where the offsets pass a multiple of 2^bits (32 bits by default;
CPA_INDEX_OFFSET_BITS lowers it so that small tensors have such points).  Whatever
the segment size and offset width, the exported index must equal the oracle's bit for
bit, and every consumer of the offsets (probes through the directory, the sampled
MTTKRP, the exact fit, the estimated fit's draws, the range finder, CP-ALS) must give
the oracle's results.
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


def _layout(monkeypatch, seg=None, bits=None, hash_tables=True):
    for name, v in (("CPA_INDEX_SEGMENT_NNZ", seg), ("CPA_INDEX_OFFSET_BITS", bits)):
        if v is None:
            monkeypatch.delenv(name, raising=False)
        else:
            monkeypatch.setenv(name, str(v))
    monkeypatch.setenv("CPA_INDEX_HASH", "1" if hash_tables else "0")


def _assert_index_equal(gi, oi, order):
    for k in range(order):
        keys, off, ik, val = cpa.cpa_index_export(gi, k)
        rk, roff, rik, rval = oi.export(k)
        np.testing.assert_array_equal(keys.cpu().numpy().astype(np.uint64), rk)
        np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), roff.astype(np.uint64))
        np.testing.assert_array_equal(ik.cpu().numpy(), rik)
        np.testing.assert_array_equal(val.cpu().numpy(), rval)


TENSORS = [
    ("3way", lambda: synth.random_sparse_tensor((60, 50, 40), 5000, seed=2)),
    ("4way", lambda: synth.random_sparse_tensor((183, 24, 1140, 1717), 30000, seed=3)),
    ("wide-keys", lambda: synth.random_sparse_tensor((2_000_000, 1_500_000, 1_800_000), 20000, seed=5)),
    ("zipf", lambda: synth.planted_cp_tensor((3000, 60, 50), 5, events=30000, seed=3, zipf_alpha=1.1)),
]


@pytest.mark.parametrize("seg,bits", [(3000, None), (700, None), (5000, 12), (1000, 12), (None, 12), (257, 13)])
@pytest.mark.parametrize("name,make", TENSORS, ids=[t[0] for t in TENSORS])
def test_segmented_index_bit_exact(monkeypatch, name, make, seg, bits):
    coo = make()
    _layout(monkeypatch, seg, bits)
    gi = cpa.cpa_index_build(coo)
    _assert_index_equal(gi, oracle.Index(coo), len(coo.dims))
    assert gi.device_bytes() > 0


def test_offset_width_too_small_is_unsupported(monkeypatch):
    coo = synth.random_sparse_tensor((60, 50, 40), 5000, seed=2)
    _layout(monkeypatch, None, 9)  # 5000 nonzeros need more than seven passes of 2^9
    with pytest.raises(cpa.CpaError) as e:
        cpa.cpa_index_build(coo)
    assert e.value.code == binding.ERR_UNSUPPORTED


def test_segments_with_empty_ranges_and_one_hot_slice(monkeypatch):
    """All nonzeros but a few in one slice of the top mode: one segment larger than
    the limit, others small or empty."""
    n = 6000
    g = np.random.default_rng(4)
    i0 = g.integers(0, 500, n).astype(np.int32)
    i1 = g.integers(0, 40, n).astype(np.int32)
    i2 = np.where(np.arange(n) < n - 50, 7, g.integers(0, 30, n)).astype(np.int32)
    key = (i2.astype(np.int64) * 40 + i1) * 500 + i0
    _, first = np.unique(key, return_index=True)
    coo = synth.Coo((500, 40, 30), [i0[first], i1[first], i2[first]], g.uniform(0.5, 2.0, first.size))
    _layout(monkeypatch, 100, 11)
    gi = cpa.cpa_index_build(coo)
    _assert_index_equal(gi, oracle.Index(coo), 3)


def test_consumers_through_directory_and_wrapped_offsets(monkeypatch):
    """Alg. 3 (FP64: factors within 1e-10 of the oracle), the exact and the estimated
    fit, the range finder and CP-ALS on an index in segments, with 12-bit stored
    offsets and no hash tables (probes through the directory)."""
    coo = synth.planted_cp_tensor((3000, 60, 50), 5, events=30000, seed=3, zipf_alpha=1.1)
    assert coo.nnz > 4 * 4096
    _layout(monkeypatch, 4000, 12, hash_tables=False)
    gi = cpa.cpa_index_build(coo)
    oi = oracle.Index(coo)
    r, s, tau, iters = 5, 2000, 1.0 / 2000, 4
    init = synth.gaussian_factors(coo.dims, r, seed=1)
    res = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=2)
    lam, fs, fit, _, _ = oracle.cp_arls_lev(oi, init, rank=r, samples=s, tau=tau, iters=iters, seed=2)
    assert max(relerr(a.cpu().numpy(), b) for a, b in zip(res.factors, fs)) < 1e-10
    assert abs(res.fit - fit) < 1e-10
    # estimated fit: the sample and its value
    gs = cpa.cpa_fit_sample(gi, 9000, alpha=0.5, seed=4)
    os_ = oracle.fit_sample(oi, 9000, alpha=0.5, seed=4)
    np.testing.assert_array_equal(gs.coords.cpu().numpy(), os_.coords)
    np.testing.assert_array_equal(gs.xs.cpu().numpy(), os_.xs)
    fit_o, F_o = oracle.fit_estimate(oi, os_, fs, lam)
    fit_g, F_g = cpa.cpa_fit_estimate(gi, gs, [torch.from_numpy(f) for f in fs], torch.from_numpy(lam))
    assert abs(F_g - F_o) <= 1e-12 * F_o
    # range finder
    om = np.random.default_rng(5).standard_normal((300, r))
    for k in range(3):
        A = cpa.cpa_rrf_init(gi, k, torch.from_numpy(om), seed=6)
        Ar = oracle.rrf_init(oi, k, om, seed=6)
        assert relerr(A.cpu().numpy(), Ar) < 1e-12
    # CP-ALS (exact MTTKRP over every fibre)
    ra = cpa.cp_als(gi, [cu(a) for a in init], rank=r, iters=2)
    la, fa, fit_a = oracle.cp_als(oi, init, rank=r, iters=2)[:3]
    assert max(relerr(a.cpu().numpy(), b) for a, b in zip(ra.factors, fa)) < 1e-10
    # mixed precision runs on it
    rm = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=2,
                         precision=binding.MIXED)
    assert abs(rm.fit - fit) < 1e-3


def _index_pair(monkeypatch, coo32, seg=None, bits=None, codes="1"):
    """(coded index, plain index) of an FP32 tensor."""
    _layout(monkeypatch, seg, bits)
    monkeypatch.setenv("CPA_INDEX_VALUE_CODES", codes)
    coded = cpa.cpa_index_build(coo32, dtype=np.float32)
    monkeypatch.setenv("CPA_INDEX_VALUE_CODES", "0")
    plain = cpa.cpa_index_build(coo32, dtype=np.float32)
    return coded, plain


@pytest.mark.parametrize("seg,bits", [(None, None), (700, 12)])
@pytest.mark.parametrize("name,make", TENSORS, ids=[t[0] for t in TENSORS])
def test_value_codes_bit_exact(monkeypatch, name, make, seg, bits):
    """FP32 values stored as 16-bit codes into a table of the distinct values: the
    exported index (values decoded) equals the oracle's, and every mode's stream is
    2 bytes per nonzero smaller."""
    coo = make().as_dtype(np.float32)
    coded, plain = _index_pair(monkeypatch, coo, seg, bits)
    _assert_index_equal(coded, oracle.Index(coo.as_dtype(np.float64)), len(coo.dims))
    nd = np.unique(coo.vals).size
    assert plain.device_bytes() - coded.device_bytes() >= 2 * coo.nnz * len(coo.dims) - 4 * nd - 4096


def test_value_codes_fall_back_with_many_distinct_values(monkeypatch):
    """More than 65,536 distinct values: stored as floats (the same index either way)."""
    g = np.random.default_rng(8)
    coo = synth.random_sparse_tensor((300, 200, 100), 90000, seed=8)
    coo = synth.Coo(coo.dims, coo.idx, g.uniform(1.0, 2.0, coo.nnz)).as_dtype(np.float32)
    assert np.unique(coo.vals).size > 65536
    coded, plain = _index_pair(monkeypatch, coo)
    assert coded.device_bytes() == plain.device_bytes()
    _assert_index_equal(coded, oracle.Index(coo.as_dtype(np.float64)), 3)


def test_consumers_with_value_codes(monkeypatch):
    """Alg. 3 in FP64 and mixed precision, the exact and estimated fit, the range
    finder and CP-ALS read coded values: the same results as from the float index
    (FP64: within 1e-12, summation order only) and the oracle's within 1e-10."""
    coo = synth.planted_cp_tensor((3000, 60, 50), 5, events=30000, seed=3, zipf_alpha=1.1).as_dtype(np.float32)
    coded, plain = _index_pair(monkeypatch, coo, 4000, 12)
    oi = oracle.Index(coo.as_dtype(np.float64))
    r, s, tau, iters = 5, 2000, 1.0 / 2000, 4
    init = synth.gaussian_factors(coo.dims, r, seed=1)
    out = {}
    for nm, gi in (("coded", coded), ("plain", plain)):
        out[nm] = cpa.cp_arls_lev(gi, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=2)
    lam, fs, fit, _, _ = oracle.cp_arls_lev(oi, init, rank=r, samples=s, tau=tau, iters=iters, seed=2)
    for a, b, c in zip(out["coded"].factors, out["plain"].factors, fs):
        assert relerr(a.cpu().numpy(), b.cpu().numpy()) < 1e-12
        assert relerr(a.cpu().numpy(), c) < 1e-10
    assert abs(out["coded"].fit - fit) < 1e-10
    gs = cpa.cpa_fit_sample(coded, 9000, alpha=0.5, seed=4)
    os_ = oracle.fit_sample(oi, 9000, alpha=0.5, seed=4)
    np.testing.assert_array_equal(gs.coords.cpu().numpy(), os_.coords)
    np.testing.assert_array_equal(gs.xs.cpu().numpy(), os_.xs)
    om = np.random.default_rng(5).standard_normal((300, r))
    A = cpa.cpa_rrf_init(coded, 1, torch.from_numpy(om), seed=6)
    assert relerr(A.cpu().numpy(), oracle.rrf_init(oi, 1, om, seed=6)) < 1e-12
    ra = cpa.cp_als(coded, [cu(a) for a in init], rank=r, iters=2)
    fa = oracle.cp_als(oi, init, rank=r, iters=2)[1]
    assert max(relerr(a.cpu().numpy(), b) for a, b in zip(ra.factors, fa)) < 1e-10
    # mixed precision: FP32 atomics make two runs differ after the first update (other
    # rounding, then other samples), so whole runs are compared with the FP64 fit
    rm = cpa.cp_arls_lev(coded, [cu(a) for a in init], rank=r, samples=s, tau=tau, iters=iters, seed=2,
                         precision=binding.MIXED)
    assert abs(rm.fit - fit) < 2e-3
