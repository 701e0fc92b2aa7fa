"""The Sec. 6.2 accuracy study through the library.

Sec. 6.2 describes the compression error (CE) over the sigma grid: very
small for small length scales (the kernel matrix is nearly diagonal and the
far field vanishes), rising to a maximum, then falling as the kernel becomes
smooth away from the diagonal.  At the paper's size (N = 1e5, d = 20,
b_k = k^-2, eta = 0.5, q = 8, the Sec. 6.2 weights, leaf 128) the float64
CE curve must peak inside the grid and start two orders of magnitude below
its peak (the paper prints 1.56e-9 at the smallest sigma and a peak of
2.75e-3; it states no leaf size, and the low end depends on it).  The
prediction errors it reports are of order 1e-3 to 1e-2 at the best
parameters; the small-size test only requires a converged solve and a
prediction error below 1.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def test_compression_error_rises_then_falls_over_sigma():
    from paper_2402_09531_gb300 import accuracy
    res = accuracy.study(n=6000, r=2.0, n_sigma=7, lambdas=[1e-3], n_cols=48, n_test=300, leaf=64,
                         maxit=1500, seed=1)
    ce = [row["ce_mean"] for row in res["rows"]]
    k = max(range(len(ce)), key=lambda i: ce[i])
    assert 0 < k < len(ce) - 1, ce            # the maximum is inside the sigma grid
    assert ce[0] < 0.1 * ce[k], ce            # nearly diagonal kernel: small far field
    assert ce[-1] < ce[k], ce
    best = min(row["pe"][1e-3]["pe"] for row in res["rows"])
    assert best < 1.0


def test_compression_error_curve_at_the_papers_size():
    """N = 1e5, d = 20, r = 2, float64, eight sigmas of the paper's log grid
    from the separation radius to the diameter, 32 random columns."""
    from paper_2402_09531_gb300 import accuracy
    res = accuracy.study(n=100000, r=2.0, n_sigma=8, n_cols=32, seed=0, precision="fp64", pe=False)
    ce = np.array([row["ce_mean"] for row in res["rows"]])
    k = int(np.argmax(ce))
    assert 0 < k < len(ce) - 1, ce
    assert ce[0] < 3e-2 * ce[k], ce
    assert ce[-1] < ce[k], ce
    assert 1e-4 < ce[k] < 1e-1, ce            # the paper's peak is 2.75e-3
