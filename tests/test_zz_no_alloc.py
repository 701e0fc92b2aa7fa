"""The allocation-free direct sum against the float64 oracle's dense product.

dwfmm_direct_sum_noalloc serves callers that cannot call cudaMalloc: a host
application whose framework owns the device memory pool (its caching
allocator has reserved nearly all of it), or a loop that cannot take the
device synchronisation that allocation implies.  It keeps all
intermediates in a fixed array inside the library.  Its result must match
the exact y = K x of the oracle's brute-force product within the float32
tolerance of the other float32 tests, on two calls in a row (the second
call reuses the array the first one left behind), up to the array's
limits (N = 8192, d = 16, 16 right-hand sides), for every kernel.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_09531_gb300 as pkg
    return pkg.lib()


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


def _case(name, n, nrhs):
    if name == "gauss_d10":
        return di.scaled(di.mixed_gauss_d10(), n, nrhs=nrhs)
    if name == "exp_d4":
        return di.scaled(di.small_exp_d4(), n, nrhs=nrhs)
    if name == "matern_d8":
        return di.scaled(di.fp64_matern_d8(), n, nrhs=nrhs)
    # d = 16 (the array's largest dimension): the serving shape, exponential kernel
    w = di.serving_requests(1)[0]
    return di.scaled(w, n, nrhs=nrhs)


@pytest.mark.parametrize("name,n,nrhs", [("gauss_d10", 1000, 16), ("exp_d4", 777, 3), ("matern_d8", 2049, 5),
                                         ("exp_d16", 8192, 16)])
def test_noalloc_matches_dense_oracle_twice(lib, name, n, nrhs):
    w = _case(name, n, nrhs)
    X, f = di.sites_and_rhs(w)
    ref = o.dense_matvec(w.kernel, X, f, w.sigma, chunk=256)
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
    st = lib.dwfmm_direct_sum_noalloc(pkg.KERNELS["exp"], 1.0, 1, 100, 4, 4, 1, 1, 17, 100, 100, None)
    assert st == 1


def test_noalloc_rejects_host_buffers(lib):
    """Host (numpy) buffers are refused on the host, before any kernel runs."""
    import torch
    import paper_2402_09531_gb300 as pkg
    w = _case("exp_d4", 300, 2)
    X, f = di.sites_and_rhs(w)
    y = np.zeros_like(f)
    Xd = torch.from_numpy(X).cuda()
    xd = torch.from_numpy(f).cuda()
    yd = torch.zeros_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    k = pkg.KERNELS[w.kernel]
    assert lib.dwfmm_direct_sum_noalloc(k, 1.0, X.ctypes.data, 300, 4, 4, xd.data_ptr(), yd.data_ptr(), 2, 300,
                                        300, s) == 1
    assert lib.dwfmm_direct_sum_noalloc(k, 1.0, Xd.data_ptr(), 300, 4, 4, f.ctypes.data, yd.data_ptr(), 2, 300,
                                        300, s) == 1
    assert lib.dwfmm_direct_sum_noalloc(k, 1.0, Xd.data_ptr(), 300, 4, 4, xd.data_ptr(), y.ctypes.data, 2, 300,
                                        300, s) == 1
    torch.cuda.synchronize()
    assert np.all(y == 0.0)
