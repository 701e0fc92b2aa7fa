"""Full-size parity: the two large workloads at their real sizes, run exactly
as bench.py runs them, compared on sampled target leaves with the float64
oracle's leaf-restricted matvec (full upward pass, far field of the leaf's
ancestors, near field), and through size-independent properties.
"""
import functools

import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


@functools.lru_cache(maxsize=None)
def _problem(name):
    w = {"fp64": di.fp64_matern_d8(), "mixed": di.mixed_gauss_d10()}[name]
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta, w.sigma)
    return w, X, f, pb


def _run(name, precision):
    import torch
    from paper_2402_09531_gb300 import Plan
    w, X, f, pb = _problem(name)
    plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta,
                leaf_size=w.leaf, precision=precision, max_rhs=w.nrhs)
    ex = plan.export_expansion()
    assert list(ex["pivots"]) == list(pb.exp_.pivots)
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    return w, X, f, pb, plan, yd.cpu().numpy()


def _sampled_err(pb, f, y, leaves):
    part = o.fmm_matvec_leaves(pb, f, leaves)
    num = den = 0.0
    worst = 0.0
    for c in leaves:
        idx = pb.tree.perm[pb.tree.begin[c]:pb.tree.end[c]]
        got = y[:, idx].T
        num += np.sum((got - part[c]) ** 2, axis=0)
        den += np.sum(part[c] ** 2, axis=0)
        worst = max(worst, float(np.max(np.abs(got - part[c]))))
    return float(np.max(np.sqrt(num / den))), worst


def test_fp64_matern_d8_full_size():
    w, X, f, pb, plan, y = _run("fp64", "fp64")
    tr = pb.tree
    first = (1 << tr.depth) - 1
    leaves = [first, first + (1 << tr.depth) // 2 + 3, tr.nclusters - 1]
    err, _ = _sampled_err(pb, f, y, leaves)
    assert err <= 1e-12
    assert plan.info()[1] == sum(len(l) for l in pb.lists.far)
    assert plan.info()[2] == len(pb.lists.near)


def test_mixed_gauss_d10_full_size_sampled():
    w, X, f, pb, plan, y = _run("mixed", "mixed")
    assert np.all(np.isfinite(y))
    tr = pb.tree
    first = (1 << tr.depth) - 1
    leaves = [first + 1234, tr.nclusters - 1]
    err, _ = _sampled_err(pb, f, y, leaves)
    assert err <= 2e-5


def test_mixed_gauss_d10_symmetry_at_full_size():
    """K_tilde is symmetric (the lists hold both orderings and the coupling
    matrices satisfy S_{t,s} = S_{s,t}^T), so u^T K_tilde v = v^T K_tilde u."""
    import torch
    w, X, f, pb, plan, y = _run("mixed", "mixed")
    u = torch.from_numpy(f[:2].copy()).cuda()
    v = torch.from_numpy(f[2:4].copy()).cuda()
    ku, kv = torch.empty_like(u), torch.empty_like(v)
    plan.matvec(u, ku)
    plan.matvec(v, kv)
    torch.cuda.synchronize()
    for r in range(2):
        a = float(torch.dot(v[r], ku[r]))
        b = float(torch.dot(u[r], kv[r]))
        scale = float(torch.linalg.norm(v[r]) * torch.linalg.norm(ku[r]))
        assert abs(a - b) <= 1e-5 * scale
