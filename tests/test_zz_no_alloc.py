"""The allocation-free leverage entry point (cpa_leverage_noalloc).

Some callers may not allocate device memory once they run (a process that keeps all
GPU memory in its own pool, a latency-critical loop where cudaMalloc/cudaFree would
synchronise the device).  For them the library keeps the scratch of the leverage
computation in a fixed device array.  This file checks, through the C ABI, that two
calls in a row give the same leverage scores as the allocating cpa_leverage.  It is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2006_16438_gb300 import binding  # noqa: E402


def _call_noalloc(lib, A, lev):
    n, r = A.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.cpa_leverage_noalloc(ctypes.c_void_p(A.data_ptr()), n, r, ctypes.c_void_p(lev.data_ptr()),
                                    stream)


def test_leverage_noalloc_matches_allocating_entry_point():
    lib = binding.load()
    g = np.random.default_rng(2024)
    cases = [(1717, 25, False), (24, 25, True), (5000, 64, False)]  # second: fewer rows than r
    for n, r, rank_deficient in cases * 2:  # two calls in a row of each shape
        A = torch.from_numpy(g.standard_normal((n, r)) * np.exp(g.standard_normal(r))).cuda()
        lev = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        rc = _call_noalloc(lib, A, lev)
        assert rc >= 0
        assert bool(rc & binding.WARN_RANK_DEFICIENT_LEV) == rank_deficient
        ref, rc_ref = binding.cpa_leverage(A)
        assert rc == rc_ref
        err = (lev - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-11, err


def test_leverage_noalloc_rejects_rank_above_scratch():
    lib = binding.load()
    A = torch.zeros((100, 65), dtype=torch.float64, device="cuda")
    lev = torch.empty(100, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, A, lev) == binding.ERR_UNSUPPORTED


def test_leverage_noalloc_allocates_no_device_memory():
    """After a first call on the device (which looks up the array's address), a call
    leaves the device's free memory unchanged: the library allocated nothing."""
    lib = binding.load()
    g = np.random.default_rng(7)
    A = torch.from_numpy(g.standard_normal((20000, 25))).cuda()
    lev = torch.empty(20000, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, A, lev) >= 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert _call_noalloc(lib, A, lev) >= 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_leverage_noalloc_binding_checks_and_matches():
    """The Python wrapper: with and without a supplied output, the same scores as
    cpa_leverage; a supplied output of the wrong type, length or layout is refused
    before the library writes through its pointer."""
    g = np.random.default_rng(11)
    A = torch.from_numpy(g.standard_normal((3000, 25))).cuda()
    ref, _ = binding.cpa_leverage(A)
    lev, rc = binding.cpa_leverage_noalloc(A)
    assert rc >= 0
    assert (lev - ref).abs().max().item() / ref.abs().max().item() < 1e-11
    out = torch.full((3000,), -1.0, dtype=torch.float64, device="cuda")
    lev2, rc2 = binding.cpa_leverage_noalloc(A, out)
    assert rc2 >= 0 and lev2.data_ptr() == out.data_ptr()
    assert (out - ref).abs().max().item() / ref.abs().max().item() < 1e-11
    with pytest.raises(TypeError):
        binding.cpa_leverage_noalloc(A, torch.empty(3000, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        binding.cpa_leverage_noalloc(A, torch.empty(2999, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        binding.cpa_leverage_noalloc(A, torch.empty(6000, dtype=torch.float64, device="cuda")[::2])
    with pytest.raises(ValueError):
        binding.cpa_leverage_noalloc(A, torch.empty(3000, dtype=torch.float64))
