"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/cpa.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cpa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for want in ("cp_arls_lev", "cpa_index_build", "cpa_skrp_lev", "cpa_sampled_mttkrp", "cpa_solve",
                 "cpa_leverage", "cpa_cdf", "cpa_fit", "cpa_philox4x64"):
        assert want in names


def test_library_exports_all_declared_symbols():
    from paper_2006_16438_gb300 import _build, binding
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == _declared()


def test_binding_has_same_names():
    import paper_2006_16438_gb300 as pkg
    for name in ("cp_arls_lev", "cpa_index_build", "cpa_skrp_lev", "cpa_sampled_mttkrp", "cpa_solve",
                 "cpa_leverage", "cpa_cdf", "cpa_fit", "cpa_philox4x64", "cp_arls_lev_coo",
                 "cpa_index_export"):
        assert callable(getattr(pkg, name))


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2006_16438_gb300 as pkg
    import synth
    with pytest.raises(RuntimeError):
        pkg.cpa_index_build(synth.random_sparse_tensor((4, 3, 2), 5))


def test_strerror_without_gpu():
    from paper_2006_16438_gb300 import binding
    lib = binding.load()
    assert lib.cpa_strerror(-5) == b"rejection limit reached in random sampling"
    opt = binding.default_options()
    assert opt.epoch_len == 5 and opt.patience == 3 and opt.reject_cap == 4096
    assert opt.tau == 2.0 ** -17 and opt.samples == 2 ** 17
    assert opt.fit_mode == binding.FIT_EXACT and opt.fit_samples == 2 ** 27 and opt.fit_alpha == 0.5
