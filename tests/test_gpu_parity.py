"""GPU path against the float64 oracle, through the C ABI.

Discrete steps (index set, pivots, tree, lists) must agree exactly; the
float64 matvec within 1e-12 relative 2-norm (worst column); the float32
matvec within FP32_TOL (derivation: each kernel entry carries a few float32
roundings, relative ~1e-7, and each of ~1e3-1e5 near-field terms per row is
summed in float32 partial sums of at most one source leaf, combined with
compensated addition, so the row error stays a small multiple of 1e-7 of the
row's absolute sum; the far field adds the float32 error of the nested
expansions, amplified by cond(V) ~ 10-100).
"""
import functools

import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _torch():
    import torch
    return torch


def _plan(w, precision="fp64", weights_rule="inv_gamma", max_rhs=16, **kw):
    from paper_2402_09531_gb300 import Plan
    return Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, weight_rule=weights_rule,
                q=w.q, eta=w.eta, leaf_size=w.leaf, precision=precision, max_rhs=max_rhs, **kw)


def _oracle_weights(w, rule):
    if rule == "inv_gamma":
        return o.weights_inv_gamma(w.gamma)
    return o.weights_paper_normalised(2.0 * w.gamma, w.eta)


@functools.lru_cache(maxsize=None)
def _oracle_problem(name, n, seed, kernel, d, q, leaf, eta, rule, nrhs):
    w = _workload(name, n, seed, kernel, d, q, leaf, eta, nrhs)
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, _oracle_weights(w, rule), w.q, w.leaf, w.eta)
    return X, f, pb


def _workload(name, n, seed, kernel, d, q, leaf, eta, nrhs):
    base = {"small": di.small_exp_d4(), "fp64": di.fp64_matern_d8(), "mixed": di.mixed_gauss_d10()}[name]
    w = di.scaled(base, n, nrhs=nrhs)
    w.seed, w.kernel, w.q, w.leaf, w.eta = seed, kernel, q, leaf, eta
    return w


def _case(name, n, seed=0, kernel=None, q=None, leaf=None, eta=1.0, rule="inv_gamma", nrhs=1):
    base = {"small": di.small_exp_d4(), "fp64": di.fp64_matern_d8(), "mixed": di.mixed_gauss_d10()}[name]
    kernel = kernel or base.kernel
    q = base.q if q is None else q
    leaf = leaf or base.leaf
    w = _workload(name, n, seed, kernel, base.d, q, leaf, eta, nrhs)
    X, f, pb = _oracle_problem(name, n, seed, kernel, base.d, q, leaf, eta, rule, nrhs)
    return w, X, f, pb


def _gpu_matvec(w, X, f, pb, precision, rule="inv_gamma", inject=True, host=False):
    torch = _torch()
    plan = _plan(w, precision, weights_rule=rule, max_rhs=max(1, f.shape[0]))
    if inject:
        plan.set_nodes(pb.exp_.nodes)
    if host:
        plan.tree_build(np.ascontiguousarray(X))
        y = np.zeros_like(f)
        plan.matvec(np.ascontiguousarray(f), y)
        return plan, y
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    return plan, yd.cpu().numpy()


# ---------------------------------------------------------------------------
# Discrete steps: exact agreement
# ---------------------------------------------------------------------------

def _near_tie_ok(A, ours, theirs):
    """First differing pick s: both candidates' residual norms at step s must
    agree to 1e-10 relative (several pivots are then equally valid)."""
    R = np.array(A, dtype=np.float64, copy=True)
    for s in range(len(ours)):
        norms = np.sum(R * R, axis=0)
        if ours[s] != theirs[s]:
            a, b = norms[ours[s]], norms[theirs[s]]
            return abs(a - b) <= 1e-10 * max(a, b)
        p = ours[s]
        qv = R[:, p] / np.sqrt(norms[p])
        R -= np.outer(qv, qv @ R)
    return True


@pytest.mark.parametrize("name,rule", [("small", "inv_gamma"), ("fp64", "inv_gamma"),
                                       ("mixed", "inv_gamma"), ("small", "paper_logrho"),
                                       ("fp64", "paper_logrho")])
def test_expansion_matches_oracle(name, rule):
    base = {"small": di.small_exp_d4(), "fp64": di.fp64_matern_d8(), "mixed": di.mixed_gauss_d10()}[name]
    plan = _plan(base, "fp64", weights_rule=rule)
    ex = plan.export_expansion()
    w = _oracle_weights(base, rule)
    np.testing.assert_allclose(ex["weights"], w, rtol=2e-16, atol=0)
    lam = o.index_set(w, base.q)
    assert np.array_equal(ex["lam"], lam)
    oe = o.make_expansion(w, base.q)
    ours, theirs = list(ex["pivots"]), list(oe.pivots)
    if ours != theirs:
        H = o.halton(o.halton_count(len(lam)), base.d)
        assert _near_tie_ok(o.basis_eval(lam, H).T, theirs, ours)
    else:
        np.testing.assert_array_equal(ex["nodes"], oe.nodes)
    V = o.basis_eval(lam, ex["nodes"])
    np.testing.assert_allclose(ex["vinv"] @ V, np.eye(len(lam)), atol=1e-10)


@pytest.mark.parametrize("n,leaf", [(4096, 64), (3001, 64), (1000, 33), (64, 64), (65, 64),
                                    (2, 2), (1, 4), (7777, 100)])
def test_tree_and_lists_match_oracle(n, leaf):
    w, X, f, pb = _case("small", n, seed=n, leaf=leaf)
    torch = _torch()
    plan = _plan(w, "fp64")
    plan.tree_build(torch.from_numpy(X).cuda())
    t = plan.export_tree()
    tr = pb.tree
    assert t["depth"] == tr.depth
    np.testing.assert_array_equal(t["perm"], tr.perm)
    np.testing.assert_array_equal(t["begin"], tr.begin)
    np.testing.assert_array_equal(t["end"], tr.end)
    np.testing.assert_array_equal(t["lo"], tr.lo)
    np.testing.assert_array_equal(t["hi"], tr.hi)
    far, near = plan.export_lists()
    ofar = np.concatenate([lvl for lvl in pb.lists.far]) if sum(len(l) for l in pb.lists.far) else np.zeros((0, 2))
    np.testing.assert_array_equal(far, ofar.astype(np.int32))
    np.testing.assert_array_equal(near, pb.lists.near.astype(np.int32))


def test_tree_with_duplicate_sites_breaks_ties_by_position():
    rng = np.random.default_rng(9)
    base = rng.random((40, 3))
    X = np.repeat(base, 25, axis=0)[rng.permutation(1000)]
    X[:100, 1] = 0.5                       # many equal coordinates
    w = di.Workload("dups", d=3, n=1000, gamma=np.ones(3), kernel="exp", q=3.0, leaf=16)
    pb = o.make_problem(X, "exp", np.ones(3), 3.0, 16, 1.0)
    torch = _torch()
    plan = _plan(w, "fp64")
    plan.tree_build(torch.from_numpy(X).cuda())
    t = plan.export_tree()
    np.testing.assert_array_equal(t["perm"], pb.tree.perm)
    far, near = plan.export_lists()
    np.testing.assert_array_equal(near, pb.lists.near.astype(np.int32))


# ---------------------------------------------------------------------------
# float64 matvec: <= 1e-12 against the oracle's FMM
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", ["exp", "matern32", "gauss"])
@pytest.mark.parametrize("n,nrhs", [(4096, 1), (3001, 3), (777, 17)])
def test_fp64_matvec_matches_oracle(kernel, n, nrhs):
    w, X, f, pb = _case("small", n, seed=1, kernel=kernel, nrhs=nrhs)
    _, y = _gpu_matvec(w, X, f, pb, "fp64")
    y_ref = o.fmm_matvec(pb, f)
    assert o.rel_err(y, y_ref) <= FP64_TOL


def test_small_workload_full_size_against_dense():
    """The d=4, N=4096 workload: GPU float64 FMM vs the oracle FMM and vs the
    dense product (compression error of the method itself)."""
    w, X, f, pb = _case("small", 4096, seed=0)
    _, y = _gpu_matvec(w, X, f, pb, "fp64", inject=False)
    y_ref = o.fmm_matvec(pb, f)
    assert o.rel_err(y, y_ref) <= FP64_TOL
    y_dense = o.dense_matvec(w.kernel, X, f)
    ce_gpu, ce_ref = o.rel_err(y, y_dense), o.rel_err(y_ref, y_dense)
    assert abs(ce_gpu - ce_ref) <= 1e-10 and ce_gpu < 0.05


def test_fp64_matvec_higher_dimension_and_weights():
    w, X, f, pb = _case("fp64", 6000, seed=3, leaf=64, nrhs=2)
    _, y = _gpu_matvec(w, X, f, pb, "fp64")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP64_TOL
    w2, X2, f2, pb2 = _case("mixed", 5000, seed=4, q=4.0, leaf=64, nrhs=2)
    _, y2 = _gpu_matvec(w2, X2, f2, pb2, "fp64")
    assert o.rel_err(y2, o.fmm_matvec(pb2, f2)) <= FP64_TOL


def test_fp64_paper_weight_rule():
    w, X, f, pb = _case("small", 2500, seed=5, rule="paper_logrho", eta=0.5)
    _, y = _gpu_matvec(w, X, f, pb, "fp64", rule="paper_logrho")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP64_TOL


@pytest.mark.parametrize("leaf,nrhs", [(128, 4), (256, 2), (128, 5)])
def test_fp64_symmetric_near_field_limits(leaf, nrhs):
    """The float64 near field evaluates each unordered near pair once when
    leaves hold <= 128 points and there are <= 4 right-hand sides (leaf 128
    with 4 RHS: both limits), and runs the list kernel otherwise (leaf 256;
    5 RHS).  Both match the oracle, and repeated matvecs are bit-identical
    (the partial sums are added in a fixed order)."""
    torch = _torch()
    w = di.Workload(f"sym_{leaf}_{nrhs}", d=3, n=2600, gamma=np.array([1.0, 0.5, 0.25]), kernel="matern32",
                    q=4.0, leaf=leaf, eta=1.0, nrhs=nrhs, seed=61)
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    plan = _plan(w, "fp64", max_rhs=nrhs)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    y1 = torch.full_like(xd, float("nan"))
    y2 = torch.full_like(xd, float("nan"))
    plan.matvec(xd, y1)
    plan.matvec(xd, y2)
    torch.cuda.synchronize()
    assert o.rel_err(y1.cpu().numpy(), o.fmm_matvec(pb, f)) <= FP64_TOL
    assert torch.equal(y1, y2)
    plan.close()


def test_host_buffers_match_device_buffers():
    w, X, f, pb = _case("small", 2000, seed=6, nrhs=2)
    _, yh = _gpu_matvec(w, X, f, pb, "fp64", host=True)
    _, yd = _gpu_matvec(w, X, f, pb, "fp64")
    np.testing.assert_array_equal(yh, yd)


@pytest.mark.parametrize("n", [1, 2, 5, 64])
def test_single_leaf_equals_dense(n):
    w, X, f, pb = _case("small", n, seed=7, nrhs=2)
    _, y = _gpu_matvec(w, X, f, pb, "fp64")
    assert o.rel_err(y, o.dense_matvec(w.kernel, X, f)) <= 1e-14


def test_empty_problem():
    torch = _torch()
    w = di.small_exp_d4()
    plan = _plan(w, "fp64")
    plan.tree_build(torch.zeros((0, 4), dtype=torch.float64, device="cuda"))
    x = torch.zeros((1, 0), dtype=torch.float64, device="cuda")
    plan.matvec(x, x.clone())
    assert plan.info()[3] == 0


def test_one_dimensional_sites():
    X = np.random.default_rng(8).random((3000, 1))
    f = np.random.default_rng(9).standard_normal((2, 3000))
    w = di.Workload("d1", d=1, n=3000, gamma=np.ones(1), kernel="exp", q=6.0, leaf=32)
    pb = o.make_problem(X, "exp", np.ones(1), 6.0, 32, 1.0)
    _, y = _gpu_matvec(w, X, f, pb, "fp64")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP64_TOL


def test_errors_and_states():
    from paper_2402_09531_gb300 import DwfmmError
    torch = _torch()
    w = di.small_exp_d4()
    plan = _plan(w, "fp64", max_rhs=2)
    x = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(DwfmmError) as e:
        plan.matvec(x, x.clone())
    assert e.value.status == 7
    X = torch.rand((10, 4), dtype=torch.float64, device="cuda")
    X[3, 2] = float("nan")
    with pytest.raises(DwfmmError) as e:
        plan.tree_build(X)
    assert e.value.status == 1
    plan.tree_build(torch.rand((10, 4), dtype=torch.float64, device="cuda"))
    x3 = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(DwfmmError) as e:
        plan.matvec(x3, x3.clone())
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# float32 matvec
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", ["exp", "matern32", "gauss"])
@pytest.mark.parametrize("n,nrhs", [(4096, 1), (3001, 16), (999, 5)])
def test_fp32_matvec_matches_oracle(kernel, n, nrhs):
    w, X, f, pb = _case("small", n, seed=2, kernel=kernel, nrhs=nrhs)
    _, y = _gpu_matvec(w, X, f, pb, "fp32")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL


def test_fp32_gauss_d10_workload_shape():
    w, X, f, pb = _case("mixed", 8192, seed=3, leaf=256, nrhs=16)
    _, y = _gpu_matvec(w, X, f, pb, "fp32")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL


# ---------------------------------------------------------------------------
# CG solve
# ---------------------------------------------------------------------------

def test_solve_fp64_residual_with_oracle_operator():
    torch = _torch()
    w, X, f, pb = _case("small", 2000, seed=11, kernel="matern32", nrhs=2)
    lam = 5.0   # K_tilde's lowest eigenvalue here is -1.34 (compression error)
    plan = _plan(w, "fp64", max_rhs=2)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    fd = torch.from_numpy(f).cuda()
    cd = torch.zeros_like(fd)
    st, its, rel = plan.solve(lam, fd, cd, rtol=1e-10, maxit=500)
    assert st == 0 and its > 0
    c = cd.cpu().numpy()
    for r in range(2):
        res = f[r] - (o.fmm_matvec(pb, c[r][None])[0] + lam * c[r])
        assert np.linalg.norm(res) / np.linalg.norm(f[r]) <= 1e-9
        assert rel[r] <= 1e-9


def test_solve_fp32_refinement_reaches_fp64_residual():
    torch = _torch()
    w, X, f, pb = _case("small", 2000, seed=12, kernel="gauss", nrhs=1)
    lam = 5.0   # K_tilde's lowest eigenvalue here is -2.03 (compression error)
    plan = _plan(w, "fp32", max_rhs=1)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    fd = torch.from_numpy(f).cuda()
    cd = torch.zeros_like(fd)
    st, its, rel = plan.solve(lam, fd, cd, rtol=1e-9, maxit=2000)
    assert st == 0
    c = cd.cpu().numpy()[0]
    res = f[0] - (o.fmm_matvec(pb, c[None])[0] + lam * c)
    assert np.linalg.norm(res) / np.linalg.norm(f[0]) <= 2e-9


def test_solve_reports_not_converged():
    torch = _torch()
    w, X, f, pb = _case("small", 1500, seed=13, kernel="exp", nrhs=1)
    plan = _plan(w, "fp64", max_rhs=1)
    plan.tree_build(torch.from_numpy(X).cuda())
    fd = torch.from_numpy(f).cuda()
    cd = torch.zeros_like(fd)
    st, its, rel = plan.solve(1e-6, fd, cd, rtol=1e-14, maxit=3)
    assert st == 5 and its == 3


def test_solve_through_negative_curvature_like_the_oracle():
    """K_tilde + 0.5 I is indefinite here (lowest eigenvalue of K_tilde -1.34,
    compression error); CG continues through negative curvature, as the
    oracle's does, and both reach the tolerance."""
    torch = _torch()
    w, X, f, pb = _case("small", 2000, seed=11, kernel="matern32", nrhs=2)
    ref = o.cg(lambda v: o.fmm_matvec(pb, v[None])[0], f[0], 0.5, 1e-8, 3000)
    assert ref.status == "ok"
    plan = _plan(w, "fp64", max_rhs=1)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    fd = torch.from_numpy(f[:1].copy()).cuda()
    cd = torch.zeros_like(fd)
    st, its, rel = plan.solve(0.5, fd, cd, rtol=1e-8, maxit=3000)
    assert st == 0
    c = cd.cpu().numpy()[0]
    res = f[0] - (o.fmm_matvec(pb, c[None])[0] + 0.5 * c)
    assert np.linalg.norm(res) / np.linalg.norm(f[0]) <= 1e-7


# ---------------------------------------------------------------------------
# MIXED plans: near field with the contraction on the tensor cores (9..16 RHS)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", ["exp", "matern32", "gauss"])
@pytest.mark.parametrize("n,nrhs,leaf", [(3001, 16, 64), (5000, 12, 256)])
def test_mixed_tensor_core_near_field_matches_oracle(kernel, n, nrhs, leaf):
    w, X, f, pb = _case("small", n, seed=31, kernel=kernel, nrhs=nrhs, leaf=leaf)
    _, y = _gpu_matvec(w, X, f, pb, "mixed")
    assert np.all(np.isfinite(y))
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL
    _, y32 = _gpu_matvec(w, X, f, pb, "fp32")
    assert o.rel_err(y, y32) <= FP32_TOL


def test_mixed_tensor_core_d10_workload_shape():
    w, X, f, pb = _case("mixed", 8192, seed=3, leaf=256, nrhs=16)
    _, y = _gpu_matvec(w, X, f, pb, "mixed")
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL


@pytest.mark.parametrize("kernel,n,leaf,nrhs,q", [("gauss", 8000, 256, 16, 4.0), ("exp", 4096, 128, 16, 4.0),
                                                    ("matern32", 8192, 256, 9, 4.0), ("gauss", 4000, 128, 12, 5.0)])
def test_mixed_symmetric_near_field_matches_oracle(kernel, n, leaf, nrhs, q):
    """Leaves of 128 or 256 slots (full or ragged: 8000 sites give 250 per
    leaf, 4000 give 125): each unordered near pair of leaves is evaluated once
    on the tensor cores (FP16 hi/lo), the transposed sums go through 64-bit
    fixed-point reductions.  Matches the oracle within the float32 tolerance,
    and repeated matvecs are bit-identical."""
    torch = _torch()
    w, X, f, pb = _case("mixed", n, seed=37, kernel=kernel, q=q, leaf=leaf, nrhs=nrhs)
    plan, y = _gpu_matvec(w, X, f, pb, "mixed")
    # the Gaussian with 256-slot leaves also takes its exponent on the tensor cores
    want = "mixed_symmetric_fp16_tensor_exponent" if (kernel == "gauss" and leaf == 256) else \
        "mixed_symmetric_fp16_tensor"
    assert plan.near_engine() == want
    assert np.all(np.isfinite(y))
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL
    xd = torch.from_numpy(f).cuda()
    y2 = torch.full_like(xd, float("nan"))
    plan.matvec(xd, y2)
    torch.cuda.synchronize()
    assert np.array_equal(y2.cpu().numpy(), y)
    plan.close()


def test_mixed_symmetric_near_field_dense_against_brute_force():
    """eta large: no admissible pair, every leaf pair is near, and the matvec
    is the exact dense product (the fp16 hi/lo split and the fixed-point
    transposed sums against the oracle's brute force)."""
    w, X, f, pb = _case("mixed", 4096, seed=38, kernel="gauss", q=2.0, leaf=256, nrhs=16, eta=1e9)
    plan, y = _gpu_matvec(w, X, f, pb, "mixed")
    assert plan.near_engine() == "mixed_symmetric_fp16_tensor_exponent"
    assert plan.info()[1] == 0
    ref = o.dense_matvec(w.kernel, X, f, w.sigma)
    assert o.rel_err(y, ref) <= FP32_TOL
    plan.close()


@pytest.mark.parametrize("sigma", [0.1, 0.35])
def test_mixed_gauss_factored_range(sigma):
    """The tensor-core near field evaluates the Gaussian as 2^(2 x'.s') with
    the factors 2^(-|x'|^2), 2^(-|s'|^2) on the sums and the charges, where
    x' = x sqrt(log2 e / (2 sigma^2)), only if |x'|^2 <= 30 on the root box.
    sigma = 0.35 is inside that range (bound ~7.8), sigma = 0.1 outside it
    (bound ~96: the CUDA-core kernel runs instead); both match the oracle."""
    torch = _torch()
    w = di.Workload(f"gauss_sigma_{sigma}", d=4, n=3001, gamma=np.array([1.0, 0.5, 0.25, 0.125]),
                    kernel="gauss", q=4.0, leaf=64, eta=1.0, nrhs=16, sigma=sigma, seed=33)
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta, w.sigma)
    plan = _plan(w, "mixed", max_rhs=16)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    assert o.rel_err(yd.cpu().numpy(), o.fmm_matvec(pb, f)) <= FP32_TOL
    plan.close()


# ---------------------------------------------------------------------------
# Tensor-product index set (Sec. 6.1's TPI) as a comparison mode
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("weights,q", [([1.0, 1.0, 1.0, 1.0], 2.0), ([1.0, 2.0, 4.0, 8.0], 4.0)])
def test_tensor_index_set_expansion_and_matvec_match_oracle(weights, q):
    from paper_2402_09531_gb300 import Plan
    torch = _torch()
    w = di.scaled(di.small_exp_d4(), 3001)
    X, f = di.sites_and_rhs(w, nrhs=2)
    wts = np.array(weights)
    plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, weight_rule="explicit", weights=wts,
                q=q, eta=w.eta, leaf_size=64, precision="fp64", max_rhs=2, index_set="tensor")
    ex = plan.export_expansion()
    lam = o.index_set(wts, q, "tensor")
    assert np.array_equal(ex["lam"], lam)
    oe = o.make_expansion(wts, q, shape="tensor")
    ours, theirs = list(ex["pivots"]), list(oe.pivots)
    if ours != theirs:
        H = o.halton(o.halton_count(len(lam)), w.d)
        assert _near_tie_ok(o.basis_eval(lam, H).T, theirs, ours)
    pb = o.make_problem(X, w.kernel, wts, q, 64, w.eta, shape="tensor")
    plan.set_nodes(pb.exp_.nodes)          # matvec parity separated from node-selection parity
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    assert o.rel_err(yd.cpu().numpy(), o.fmm_matvec(pb, f)) <= FP64_TOL
    plan.close()


@pytest.mark.parametrize("d,kernel,n_sites", [(7, "matern32", 2600), (12, "gauss", 2600), (15, "exp", 2400),
                                              (20, "gauss", 2000)])
def test_mixed_tensor_core_every_padded_dimension(d, kernel, n_sites):
    """The tensor-core engine is instantiated for padded dimensions 4, 8, 10,
    12, 16 and 20 (d = 7 pads to 8, 15 to 16): each of those not covered by
    the workload shapes against the oracle, 16 right-hand sides, leaves of 256
    (two 128-target tiles per leaf) and a ragged count."""
    from paper_2402_09531_gb300 import Plan
    torch = _torch()
    w = di.Workload(f"dims_{d}", d=d, n=n_sites, gamma=di.gamma_inverse_square(d), kernel=kernel, q=2.0,
                    leaf=256, eta=1.0, nrhs=16, seed=40 + d)
    X, f = di.sites_and_rhs(w)
    wts = o.weights_inv_gamma(w.gamma)
    pb = o.make_problem(X, kernel, wts, w.q, w.leaf, w.eta)
    plan = Plan(d=d, kernel=kernel, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf, precision="mixed",
                max_rhs=16)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    assert o.rel_err(yd.cpu().numpy(), o.fmm_matvec(pb, f)) <= FP32_TOL
    plan.close()
