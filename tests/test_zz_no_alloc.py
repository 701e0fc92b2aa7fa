"""The allocation-free direct sum against the library's own exact path.

dwfmm_direct_sum_noalloc serves callers that cannot call cudaMalloc (their
framework owns the device memory pool, or their loop cannot take the device
synchronisation that allocation implies); it keeps all intermediates in a
fixed array inside the library.  Its result must match what dwfmm_matvec
gives for the same sites when the whole set fits in one leaf (then the FMM
has no far field and is the exact direct sum), within the float32 tolerance
used by the other float32 tests, on two calls in a row (the second call
reuses the array the first one left behind).

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import dwfmm_inputs as di

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_09531_gb300 as pkg
    return pkg.lib()


def _reference(w, X, f):
    import torch
    from paper_2402_09531_gb300 import Plan
    plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta,
                leaf_size=1024, precision="fp32", max_rhs=f.shape[0])
    plan.tree_build(torch.from_numpy(X).cuda())
    assert plan.info()[3] == 0            # one leaf: the matvec is the exact sum
    xd = torch.from_numpy(f).cuda()
    yd = torch.empty_like(xd)
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _noalloc(lib, w, X, f):
    import torch
    import paper_2402_09531_gb300 as pkg
    Xd = torch.from_numpy(X).cuda()
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    st = lib.dwfmm_direct_sum_noalloc(pkg.KERNELS[w.kernel], w.sigma, Xd.data_ptr(), X.shape[0], X.shape[1],
                                      Xd.stride(0), xd.data_ptr(), yd.data_ptr(), f.shape[0], xd.stride(0),
                                      yd.stride(0), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("base,n,nrhs", [("mixed", 1000, 16), ("small", 777, 3)])
def test_noalloc_matches_single_leaf_matvec_twice(lib, base, n, nrhs):
    w = di.scaled({"mixed": di.mixed_gauss_d10(), "small": di.small_exp_d4()}[base], n, nrhs=nrhs)
    X, f = di.sites_and_rhs(w)
    ref = _reference(w, X, f)
    first = _noalloc(lib, w, X, f)
    second = _noalloc(lib, w, X, f)
    assert np.all(np.isfinite(first)) and np.all(np.isfinite(second))
    assert _rel(first, ref) <= FP32_TOL
    assert _rel(second, ref) <= FP32_TOL


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    import paper_2402_09531_gb300 as pkg
    st = lib.dwfmm_direct_sum_noalloc(pkg.KERNELS["exp"], 1.0, 1, 8193, 4, 4, 1, 1, 1, 8193, 8193, None)
    assert st == 1
    st = lib.dwfmm_direct_sum_noalloc(pkg.KERNELS["exp"], 1.0, 1, 100, 17, 17, 1, 1, 1, 100, 100, None)
    assert st == 1
