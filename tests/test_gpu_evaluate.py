"""Evaluation of the kernel interpolant at new points (Sec. 2; the
prediction error of Sec. 6.2 evaluates it at test points), and the d=20
shape of the Sec. 6.2 study, against the oracle."""
import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _plan(w, precision, rule="inv_gamma", max_rhs=16):
    from paper_2402_09531_gb300 import Plan
    return Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, weight_rule=rule, q=w.q, eta=w.eta,
                leaf_size=w.leaf, precision=precision, max_rhs=max_rhs)


@pytest.mark.parametrize("precision,base,n,nt,nrhs,tol", [
    ("fp64", "small", 3001, 300, 2, 1e-12),
    ("fp32", "small", 3001, 777, 3, 2e-5),
    ("fp32", "mixed", 5000, 1000, 16, 2e-5),
])
def test_evaluate_matches_dense_oracle(precision, base, n, nt, nrhs, tol):
    import torch
    w = di.scaled({"small": di.small_exp_d4(), "mixed": di.mixed_gauss_d10()}[base], n, nrhs=nrhs)
    X, c = di.sites_and_rhs(w)
    rng = np.random.default_rng(123)
    T = (2 * rng.random((nt, w.d)) - 1) * w.gamma[None, :]
    plan = _plan(w, precision, max_rhs=nrhs)
    plan.tree_build(torch.from_numpy(X).cuda())
    out = torch.full((nrhs, nt), float("nan"), dtype=torch.float64, device="cuda")
    plan.evaluate(torch.from_numpy(T).cuda(), torch.from_numpy(c).cuda(), out)
    ref = (o.kernel_matrix(w.kernel, T, X, w.sigma) @ c.T).T
    assert o.rel_err(out.cpu().numpy(), ref) <= tol
    # host buffers give the same numbers
    out_h = np.zeros((nrhs, nt))
    plan.evaluate(T, c, out_h)
    np.testing.assert_array_equal(out_h, out.cpu().numpy())


def test_d20_study_shape_matvec_and_evaluate():
    """Sec. 6.2 shape: d=20, sites scaled by b_k = k^-2, exponential kernel,
    eta=0.5, q=8, the Sec. 6.2 weight rule (float32)."""
    import torch
    n, d = 3000, 20
    b = np.array([1.0 / (k * k) for k in range(1, d + 1)])
    w = di.Workload("s62", d=d, n=n, gamma=b / 2.0, kernel="exp", q=8.0, leaf=64, eta=0.5, seed=21, nrhs=2)
    X, c = di.sites_and_rhs(w)
    pb = o.make_problem(X, "exp", o.weights_paper_normalised(b, 0.5), 8.0, 64, 0.5)
    plan = _plan(w, "fp32", rule="paper_logrho", max_rhs=2)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    y = torch.empty((2, n), dtype=torch.float64, device="cuda")
    plan.matvec(torch.from_numpy(c).cuda(), y)
    torch.cuda.synchronize()
    assert o.rel_err(y.cpu().numpy(), o.fmm_matvec(pb, c)) <= 2e-5
    T = (2 * np.random.default_rng(5).random((500, d)) - 1) * w.gamma[None, :]
    out = np.zeros((2, 500))
    plan.evaluate(T, c, out)
    assert o.rel_err(out, (o.kernel_matrix("exp", T, X) @ c.T).T) <= 2e-5
