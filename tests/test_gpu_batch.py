"""Batches: many uneven problems (the batching workload's generator: N
log-uniform in [2048, 65536], d in {6..12}, gamma_k = k^-2, Matern-3/2, q=5,
1-8 right-hand sides) in one fused matvec.  Every problem's result must equal
its own single-problem matvec (same kernels, the padded coordinates and
charges contribute exact zeros), and the oracle's FMM on small problems."""
import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _setup(count, nmax):
    import torch
    from paper_2402_09531_gb300 import Plan
    probs = [w for w in di.batching_problems(256) if w.n <= nmax][:count]
    plans, xs, ys, data = [], [], [], []
    for w in probs:
        X, f = di.sites_and_rhs(w)
        p = Plan(d=w.d, kernel=w.kernel, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf, precision="fp32",
                 max_rhs=w.nrhs)
        p.tree_build(torch.from_numpy(X).cuda())
        plans.append(p)
        xs.append(torch.from_numpy(f).cuda())
        ys.append(torch.full_like(xs[-1], float("nan")))
        data.append((w, X, f))
    return probs, plans, xs, ys, data


def test_batch_equals_single_problem_matvecs():
    import torch
    from paper_2402_09531_gb300 import Batch
    probs, plans, xs, ys, data = _setup(24, 12000)
    assert len(set(w.nrhs for w in probs)) > 2 and len(set(w.d for w in probs)) > 2
    b = Batch(plans, [w.nrhs for w in probs])
    b.matvec(xs, ys)
    torch.cuda.synchronize()
    info = b.info()
    assert info["leaves"] == sum(p.info()[3] >= 0 and 2 ** p.info()[3] for p in plans)
    # the autotuner picked one timed shape for each fused launch
    for k in ("near_shape", "m2l_shape"):
        assert info[k]["threads"] in (32, 64, 96, 128), info
    assert info["split"] == info["near_shape"]["per_class"]
    assert 0 < min(info["tune_ms"])
    for i, p in enumerate(plans):
        ref = torch.empty_like(xs[i])
        p.matvec(xs[i], ref)
        torch.cuda.synchronize()
        got, want = ys[i].cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert o.rel_err(got, want) <= 1e-6
    # a second call through the same graph gives the same answer
    ys2 = [torch.full_like(x, float("nan")) for x in xs]
    b.matvec(xs, ys2)
    torch.cuda.synchronize()
    for y1, y2 in zip(ys, ys2):
        assert torch.equal(y1, y2)
    b.close()


def test_batch_matches_oracle_on_small_problems():
    import torch
    from paper_2402_09531_gb300 import Batch
    probs, plans, xs, ys, data = _setup(6, 4000)
    b = Batch(plans, [w.nrhs for w in probs])
    b.matvec(xs, ys)
    torch.cuda.synchronize()
    for i in (0, len(probs) - 1):
        w, X, f = data[i]
        pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
        assert o.rel_err(ys[i].cpu().numpy(), o.fmm_matvec(pb, f)) <= FP32_TOL
    b.close()


def test_persistent_engine_equals_launch_graph():
    """The whole batch matvec as one persistent cooperative launch (phases
    separated by grid-wide barriers, near-field groups taken from a work queue
    while the far-field phases wait) sums every target in the order of the
    captured launches: both engines give the same result bit for bit, on
    repeated calls, and in batched CG iterations."""
    import torch
    from paper_2402_09531_gb300 import Batch
    probs, plans, xs, ys, data = _setup(24, 12000)
    b = Batch(plans, [w.nrhs for w in probs])
    b.set_engine("persistent")      # tunes the persistent engine if creation did not
    e = b.engine()
    assert e["persistent_available"] and e["engine"] == "persistent", e
    assert e["ms"]["graph"] > 0 and e["ms"]["persistent"] > 0, e
    launch = e["persistent_launch"]
    assert launch["ctas"] > 0 and launch["near_threads"] in (32, 64, 128) and launch["m2l_threads"] in (32, 64, 128)
    results = {}
    for eng in ("graph", "persistent", "graph", "persistent"):
        b.set_engine(eng)
        assert b.engine()["engine"] == eng
        out = [torch.full_like(x, float("nan")) for x in xs]
        b.matvec(xs, out)
        torch.cuda.synchronize()
        if eng in results:
            for y1, y2 in zip(results[eng], out):
                assert torch.equal(y1, y2)
        results[eng] = out
    for i, (yg, yp) in enumerate(zip(results["graph"], results["persistent"])):
        assert torch.isfinite(yp).all(), i
        assert torch.equal(yg, yp), (i, float((yg - yp).abs().max()))
    # the oracle on the smallest problem
    k = min(range(len(probs)), key=lambda i: probs[i].n)
    w, X, f = data[k]
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta)
    assert o.rel_err(results["persistent"][k].cpu().numpy(), o.fmm_matvec(pb, f)) <= FP32_TOL
    # batched CG: same iterates with either engine
    lam = 1e-1
    sols = {}
    for eng in ("graph", "persistent"):
        b.set_engine(eng)
        for p, x in zip(plans, xs):
            p.cg_begin(lam, x, rtol=1e-6)
        b.cg_step(12)
        torch.cuda.synchronize()
        cs = []
        for p, x in zip(plans, xs):
            c = torch.empty_like(x)
            p.cg_result(c)
            cs.append(c)
        torch.cuda.synchronize()
        sols[eng] = cs
    for c1, c2 in zip(sols["graph"], sols["persistent"]):
        assert torch.equal(c1, c2)
    b.close()
