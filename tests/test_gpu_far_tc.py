"""Expansion phases of MIXED plans on the tensor cores (Sec. 5.2, Eq. (5.4)):
P2M, M2M, L2L and L2P as per-cluster contractions with FP16 hi/lo basis
values and right-hand sides, and the V^{-T} / V^{-1} transforms as one GEMM
per tree level.  Each case must take that engine, match the oracle's FMM
within the float32 tolerance and the float64 GPU matvec of the same plan
parameters far tighter (the hi/lo split carries ~2^-22 relative per
element, the level of the float32 CUDA-core path), repeat bit-identically,
and handle ragged leaves, fewer than 16 right-hand sides and several
16-column passes.  These cases force the symmetric M2L (each unordered far
pair once) where it applies; the last test checks the timed default."""
import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5
# against float64 with the same nodes and tree: the near field's float32
# evaluation dominates (~1e-6 worst column at these sizes)
VS_FP64_TOL = 5e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _run(w, X, f, pb, precision, m2l="mixed_symmetric_fp16_tensor"):
    import torch
    from paper_2402_09531_gb300 import Plan
    plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf,
                precision=precision, max_rhs=max(1, f.shape[0]))
    plan.set_m2l_engine(m2l)
    plan.set_nodes(pb.exp_.nodes)
    plan.tree_build(torch.from_numpy(X).cuda())
    xd = torch.from_numpy(f).cuda()
    yd = torch.full_like(xd, float("nan"))
    plan.matvec(xd, yd)
    torch.cuda.synchronize()
    return plan, xd, yd


def _worst_col(a, b):
    return max(o.rel_err(a[i], b[i]) for i in range(a.shape[0]))


@pytest.mark.parametrize("base,n,leaf,nrhs,q,eta,seed", [
    ("mixed", 12000, 256, 16, 8.0, 0.6, 51),   # the d = 10 Gaussian shape (|Lambda| = 116), ragged leaves
    ("mixed", 6000, 128, 5, 6.0, 0.5, 52),     # 5 right-hand sides, eta = 0.5: more far field
    ("small", 9000, 128, 20, 4.0, 1.0, 53),    # d = 4 exponential, two passes (16 + 4 columns)
    ("fp64", 7000, 256, 12, 8.0, 0.7, 54),     # d = 8 Matern-3/2
])
def test_tensor_core_far_field_matches_oracle_and_fp64(base, n, leaf, nrhs, q, eta, seed):
    import torch
    b = {"small": di.small_exp_d4(), "fp64": di.fp64_matern_d8(), "mixed": di.mixed_gauss_d10()}[base]
    w = di.scaled(b, n, nrhs=nrhs)
    w.leaf, w.q, w.eta, w.seed = leaf, q, eta, seed
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    assert len(pb.exp_.nodes) <= 128
    plan, xd, yd = _run(w, X, f, pb, "mixed")
    assert plan.far_engine() == "mixed_fp16_tensor"
    assert plan.info()[1] > 0            # the far field is not empty
    # a pass of 9..16 right-hand sides: each unordered far pair once (M2L);
    # the engine reported is the last pass's
    last = nrhs % 16 or 16
    assert plan.m2l_engine() == ("mixed_symmetric_fp16_tensor" if last >= 9 else "fp32_cuda_cores")
    y = yd.cpu().numpy()
    assert np.all(np.isfinite(y))
    assert o.rel_err(y, o.fmm_matvec(pb, f)) <= FP32_TOL
    p64, _, y64 = _run(w, X, f, pb, "fp64")
    assert p64.far_engine() == "fp64_cuda_cores"
    assert _worst_col(y, y64.cpu().numpy()) <= VS_FP64_TOL
    y2 = torch.full_like(xd, float("nan"))
    plan.matvec(xd, y2)
    torch.cuda.synchronize()
    assert torch.equal(y2, yd)
    plan.close()
    p64.close()


def test_far_field_engines_by_plan():
    """Leaves of 64 sites keep the float32 CUDA-core expansions in a MIXED
    plan, float32 plans always do; both match the oracle."""
    w = di.scaled(di.small_exp_d4(), 3000, nrhs=16)
    w.seed = 55
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    for prec in ("mixed", "fp32"):
        plan, _, yd = _run(w, X, f, pb, prec)
        assert plan.far_engine() == "fp32_cuda_cores"
        assert o.rel_err(yd.cpu().numpy(), o.fmm_matvec(pb, f)) <= FP32_TOL
        plan.close()


def test_far_field_alone_against_oracle_expansion():
    """A right-hand side that is zero on every leaf near a target block
    leaves only far-field contributions in those rows: they must match the
    oracle's far field to the float32 tolerance (the near field cannot hide
    an error of the expansions)."""
    b = di.mixed_gauss_d10()
    w = di.scaled(b, 8192, nrhs=16)
    w.seed, w.eta = 56, 0.6
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    # zero the charges of every leaf that is near leaf 0; keep the others
    t = pb.tree
    leaf0 = (1 << t.depth) - 1
    near = pb.lists.near
    near0 = [int(s) for s in near[near[:, 0] == leaf0][:, 1]]
    assert leaf0 in near0
    f2 = f.copy()
    for c in near0:
        f2[:, t.perm[t.begin[c]:t.end[c]]] = 0.0
    rows = t.perm[t.begin[leaf0]:t.end[leaf0]]
    plan, _, yd = _run(w, X, f2, pb, "mixed")
    assert plan.far_engine() == "mixed_fp16_tensor"
    y = yd.cpu().numpy()[:, rows].T
    ref = o.fmm_matvec_leaves(pb, f2, [leaf0])[leaf0]
    assert np.linalg.norm(ref) > 0
    assert o.rel_err(y, ref) <= FP32_TOL
    plan.close()


@pytest.mark.parametrize("leaf,n", [(256, 5000), (128, 6000)])
def test_m2l_engines_agree_and_the_default_is_timed(leaf, n):
    """Both tensor-core M2L engines (every ordered far pair; each unordered
    pair once) match the oracle; the default times both at the first
    matvec of the tree and runs the faster, reporting the two times.  The
    first case has far blocks at a coarse level (jmin = 3 of 5) whose
    parents never get moments."""
    b = di.small_exp_d4()
    w = di.scaled(b, n, nrhs=16)
    w.seed, w.leaf = 57, leaf
    X, f = di.sites_and_rhs(w)
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    ref = o.fmm_matvec(pb, f)
    outs = {}
    for eng in ("mixed_tf32_tensor", "mixed_symmetric_fp16_tensor", "auto"):
        plan, _, yd = _run(w, X, f, pb, "mixed", m2l=eng)
        got = plan.m2l_engine()
        if eng == "auto":
            ms = plan.m2l_tune_ms()
            assert ms[0] > 0 and ms[1] > 0, ms
            assert got == ("mixed_symmetric_fp16_tensor" if ms[0] < ms[1] else "mixed_tf32_tensor")
        else:
            assert got == eng
        outs[eng] = yd.cpu().numpy()
        assert o.rel_err(outs[eng], ref) <= FP32_TOL
        plan.close()
    assert o.rel_err(outs["mixed_tf32_tensor"], outs["mixed_symmetric_fp16_tensor"]) <= 2 * FP32_TOL
