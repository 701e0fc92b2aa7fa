"""Host-side checks of the C-ABI library (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/dwfmm.h declares; argument validation that happens before any CUDA
call must reject bad configurations.
"""
import ctypes as C
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dwfmm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dwfmm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2402_09531_gb300 import build as b
    b.build()
    import paper_2402_09531_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("dwfmm_plan_create", "dwfmm_tree_build", "dwfmm_matvec", "dwfmm_solve",
                 "dwfmm_plan_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2402_09531_gb300 as pkg
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    assert sorted(pkg.EXPORTS) == names


def test_status_strings(lib):
    for s in range(9):
        assert lib.dwfmm_status_string(s)
    assert b"breakdown" in lib.dwfmm_status_string(4)


def _cfg(pkg, **kw):
    g = np.ones(4)
    base = dict(d=4, kernel=0, sigma=1.0, gamma=g.ctypes.data_as(C.POINTER(C.c_double)),
                weight_rule=0, weights=None, q=4.0, eta=1.0, leaf_size=64,
                halton_candidates=0, precision=0, max_rhs=4)
    base.update(kw)
    return pkg.dwfmm.dwfmm_config(**base), g


@pytest.mark.parametrize("bad", [dict(d=0), dict(d=33), dict(kernel=7), dict(sigma=0.0),
                                 dict(q=-1.0), dict(eta=0.0), dict(leaf_size=1),
                                 dict(leaf_size=4096), dict(precision=5), dict(max_rhs=0),
                                 dict(weight_rule=2), dict(gamma=None)])
def test_invalid_config_rejected_before_any_cuda_call(lib, bad):
    import paper_2402_09531_gb300 as pkg
    cfg, keep = _cfg(pkg, **bad)
    h = C.c_void_p()
    st = lib.dwfmm_plan_create(C.byref(cfg), None, C.byref(h))
    assert st == 1 and not h.value


def test_null_plan_is_rejected(lib):
    assert lib.dwfmm_matvec(None, None, None, 1, 1, 1, None) == 1
    assert lib.dwfmm_plan_destroy(None) == 0
    assert lib.dwfmm_last_error(None) == b""


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2402_09531_gb300 import dwfmm
    with pytest.raises(ImportError):
        dwfmm.load(str(tmp_path / "missing.so"))


def test_binding_rejects_buffers_the_abi_would_misread():
    """Every (R, N) / (N, d) buffer crosses the C ABI as a pointer plus a row
    stride of float64 elements; the binding refuses any other layout before
    a call is made."""
    import torch
    from paper_2402_09531_gb300.dwfmm import _ld, _same_layout
    assert _ld(np.zeros((3, 10)), "a") == 10
    assert _ld(np.zeros((4, 12))[:, :10], "a") == 12
    assert _ld(torch.zeros((2, 7), dtype=torch.float64), "t") == 7
    assert _ld(torch.zeros((1, 0), dtype=torch.float64), "t") >= 0
    bad = [np.zeros((3, 10), dtype=np.float32), np.zeros(10), np.zeros((10, 3)).T,
           torch.zeros((2, 3)), torch.zeros((3, 2), dtype=torch.float64).t(),
           torch.zeros(5, dtype=torch.float64)]
    for b in bad:
        with pytest.raises(ValueError):
            _ld(b, "b")
    f = np.zeros((2, 5))
    _same_layout(f, "f", 5, (np.zeros((2, 5)), "c"), (None, "r"))
    with pytest.raises(ValueError):
        _same_layout(f, "f", 5, (np.zeros((2, 6))[:, :5], "c"))
    with pytest.raises(ValueError):
        _same_layout(f, "f", 5, (np.zeros((3, 5)), "c"))
