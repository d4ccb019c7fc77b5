"""The planted-tensor generator used for the billion-nonzero workloads, run on the
host device at small sizes: coordinates unique, in range and in ascending
(i_0, ..., i_{d-1}) order; counts sum to the events drawn; log(1 + count) values;
the same output for the same seed.  (Input generation only: none of the method's
arithmetic.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import gpu as sgpu  # noqa: E402


def _gen(dims, events, seed, log_counts=False, per_slice=1 << 12):
    idx, vals = sgpu.planted_cp_tensor_gpu(dims, 5, events=events, seed=seed, zipf_alpha=1.2, log_counts=log_counts,
                                           events_per_slice=per_slice, device="cpu")
    return [i.numpy().astype(np.int64) for i in idx], vals.numpy()


@pytest.mark.parametrize("dims", [(300, 40, 250), (50, 20, 30, 40)])
def test_coordinates_unique_sorted_in_range_and_counts_sum_to_events(dims):
    events = 30000
    idx, vals = _gen(dims, events, seed=3)
    n = vals.size
    assert n > 0 and all(i.size == n for i in idx)
    for i, d in zip(idx, dims):
        assert i.min() >= 0 and i.max() < d
    lin = np.zeros(n, dtype=np.int64)
    for i, d in zip(idx, dims):
        lin = lin * d + i
    assert np.all(np.diff(lin) > 0)  # unique and ascending, i_0 most significant
    assert np.all(vals >= 1) and np.all(vals == np.round(vals))
    assert int(vals.sum()) == events


def test_log_counts_and_determinism():
    dims = (200, 30, 150)
    idx_a, counts = _gen(dims, 20000, seed=5)
    idx_b, logv = _gen(dims, 20000, seed=5, log_counts=True)
    for a, b in zip(idx_a, idx_b):
        np.testing.assert_array_equal(a, b)
    # float32 log(1 + count) of the same counts (libraries may round the last bit
    # differently, so compare the counts it encodes and the value to one ulp)
    np.testing.assert_array_equal(np.rint(np.expm1(logv.astype(np.float64))), counts)
    np.testing.assert_allclose(logv, np.log1p(counts.astype(np.float64)), rtol=1.2e-7, atol=0)
    idx_c, _ = _gen(dims, 20000, seed=6)
    assert any(a.size != c.size or np.any(a != c) for a, c in zip(idx_a, idx_c))
