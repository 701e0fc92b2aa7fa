"""Serving: many CG solves in flight on one GPU (continuous batching).

Each served result must be the same alone and in the mix (every request
owns its plan, stream and Krylov state; reductions have a fixed order, so
the results are bit-identical), admission must respect the memory budget,
the incremental device-side CG must agree with the blocking solve, and the
served solutions must meet the tolerance with the oracle's operator.

Serving workload (Sec. 6.2 style sites, the serving generator): d=16,
gamma_k=2^-k, exponential kernel, q=6, lambda=1e-6, rtol=1e-6.  Readings for
the unstated parameters: eta=2 and the Sec. 6.2 weight rule, leaf 128 (with
eta=1 or the gamma_1/gamma_k weights the compressed matrix has eigenvalues
below -0.1 at these sizes and CG breaks down for lambda=1e-6, in the oracle
as well).
"""
import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def _requests(ns, seed0=50, arrival=0.0):
    from paper_2402_09531_gb300.serving import Request
    out = []
    for i, n in enumerate(ns):
        w = di.Workload(f"r{i}", d=16, n=n, gamma=di.gamma_half_powers(16), kernel="exp", q=6.0, leaf=128,
                        eta=2.0, seed=seed0 + i)
        X, f = di.sites_and_rhs(w, nrhs=1)
        out.append(Request(rid=i, X=X, f=f, kernel="exp", gamma=w.gamma, q=6.0, eta=2.0, leaf=128,
                           weight_rule="paper_logrho", lam=1e-6, rtol=1e-6, maxit=4000, arrival=arrival * i))
    return out


def test_same_result_alone_and_in_the_mix():
    from paper_2402_09531_gb300.serving import Server
    reqs = _requests([1500, 2600, 900, 3200, 2000, 1200])
    alone = Server(precision="fp32", max_active=1)
    r_alone = alone.run([reqs[0]])[0]
    alone.close()
    mix = Server(precision="fp32", max_active=6)
    res = {r.rid: r for r in mix.run(reqs)}
    assert mix.peak_active >= 4
    mix.close()
    assert r_alone.status == "ok"
    assert res[0].status == "ok" and res[0].iters == r_alone.iters
    np.testing.assert_array_equal(res[0].c, r_alone.c)
    for rid in (1, 3):
        r = reqs[rid]
        pb = o.make_problem(r.X, "exp", o.weights_paper_normalised(2 * r.gamma, 2.0), 6.0, 128, 2.0)
        c = res[rid].c[0]
        resid = r.f[0] - (o.fmm_matvec(pb, c[None])[0] + r.lam * c)
        assert res[rid].status == "ok"
        assert np.linalg.norm(resid) / np.linalg.norm(r.f[0]) <= 2e-6


def test_admission_respects_memory_budget():
    from paper_2402_09531_gb300.serving import Server, estimate_bytes
    reqs = _requests([1000, 1100, 1200], seed0=70)
    one = estimate_bytes(1200, 16, 1, 128, 0)
    srv = Server(precision="fp32", max_active=8, mem_budget=one + 1)
    res = srv.run(reqs)
    assert srv.peak_active == 1 and len(res) == 3
    srv.close()


def test_incremental_cg_matches_blocking_solve():
    import torch
    from paper_2402_09531_gb300 import Plan
    w = di.scaled(di.small_exp_d4(), 2000, nrhs=2)
    w.kernel = "matern32"
    X, f = di.sites_and_rhs(w)
    kw = dict(d=4, kernel="matern32", gamma=w.gamma, q=4.0, eta=1.0, leaf_size=64, precision="fp64", max_rhs=2)
    fd = torch.from_numpy(f).cuda()
    a = Plan(**kw)
    a.tree_build(torch.from_numpy(X).cuda())
    ca = torch.zeros_like(fd)
    st, its, rel = a.solve(5.0, fd, ca, rtol=1e-10, maxit=500)
    assert st == 0
    b = Plan(**kw)
    b.tree_build(torch.from_numpy(X).cuda())
    b.cg_begin(5.0, fd, rtol=1e-10)
    for _ in range(200):
        b.cg_step(5)
        torch.cuda.synchronize()
        ready, status, iters, rr = b.cg_poll()
        assert ready
        if np.all(status != 0):
            break
    assert np.all(status == 1)
    cb = torch.zeros_like(fd)
    b.cg_result(cb)
    torch.cuda.synchronize()
    assert int(iters.max()) == its
    np.testing.assert_allclose(cb.cpu().numpy(), ca.cpu().numpy(), rtol=0, atol=1e-12 * float(ca.abs().max()))


def _run_incremental(plan, lam, fd, steps, stream, rtol=1e-10, rounds=400):
    """Incremental CG on `stream` with the given iteration counts per step
    (cycled); returns (status, iters, c)."""
    import torch
    with torch.cuda.stream(stream):
        plan.cg_begin(lam, fd, rtol=rtol, stream=stream)
        for k in range(rounds):
            plan.cg_step(steps[k % len(steps)], stream=stream)
            stream.synchronize()
            ready, status, iters, rr = plan.cg_poll()
            assert ready
            if np.all(status != 0):
                break
        c = torch.zeros_like(fd)
        plan.cg_result(c, stream=stream)
        stream.synchronize()
    return status, iters, c.cpu().numpy()


@pytest.mark.parametrize("precision,nrhs,rtol", [("fp64", 2, 1e-10), ("mixed", 16, 1e-5)])
def test_captured_cg_iterations_equal_plain_launches(precision, nrhs, rtol):
    """cg_step replays a captured CUDA graph of its iterations from the second
    step with the same configuration on a non-default stream.  Constant step
    sizes take that path; alternating step sizes never do (every step starts a
    new configuration).  Both must give the same solution bit for bit, also
    after the tree is rebuilt on other sites (the graph must not be reused)."""
    import torch
    from paper_2402_09531_gb300 import Plan
    w = di.scaled(di.mixed_gauss_d10(), 3000, nrhs=nrhs)
    X, f = di.sites_and_rhs(w)
    X2 = X[::-1].copy() * 0.9
    kw = dict(d=w.d, kernel=w.kernel, gamma=w.gamma, q=4.0, eta=1.0, leaf_size=64, precision=precision,
              max_rhs=nrhs)
    s = torch.cuda.Stream()
    fd = torch.from_numpy(f).cuda()
    torch.cuda.synchronize()
    results = []
    for steps in ([5], [4, 6]):
        p = Plan(**kw)
        out = []
        for pts in (X, X2):
            with torch.cuda.stream(s):
                p.tree_build(torch.from_numpy(pts).cuda(), stream=s)
            st, its, c = _run_incremental(p, 2.0, fd, steps, s, rtol=rtol)
            assert np.all(st == 1)
            out.append(c)
        results.append(out)
        p.close()
    for a, b in zip(*results):
        assert np.array_equal(a, b)
    # and a fresh plan on the second tree agrees with the rebuilt one
    q = Plan(**kw)
    with torch.cuda.stream(s):
        q.tree_build(torch.from_numpy(X2).cuda(), stream=s)
    _, _, c2 = _run_incremental(q, 2.0, fd, [5], s, rtol=rtol)
    assert np.array_equal(c2, results[0][1])
    q.close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_refine_step_never_raises_the_float64_residual(precision):
    """dwfmm_refine: with a useless correction the float64 residual does not
    grow (the step length shrinks instead), the updated residual equals
    f - (K64 + lam I) c recomputed from scratch, and with the float64
    solution as correction the step length is ~1 and the residual vanishes."""
    import torch
    from paper_2402_09531_gb300 import Plan
    w = di.scaled(di.small_exp_d4(), 2000, nrhs=2)
    X, f = di.sites_and_rhs(w)
    lam = 0.5
    kw = dict(d=4, kernel=w.kernel, gamma=w.gamma, q=4.0, eta=1.0, leaf_size=64, max_rhs=2)
    p = Plan(precision=precision, **kw)
    p.tree_build(torch.from_numpy(X).cuda())
    fd = torch.from_numpy(f).cuda()
    c = torch.zeros_like(fd)
    r = fd.clone()
    junk = torch.from_numpy(np.random.default_rng(9).standard_normal(f.shape) * 1e3).cuda()
    alpha, rel = p.refine(lam, fd, c, junk, r)
    assert np.all(rel <= 1.0 + 1e-12)
    rel_true = p.residual(lam, fd, c)
    np.testing.assert_allclose(rel, rel_true, rtol=1e-9)
    p64 = Plan(precision="fp64", **kw)
    p64.tree_build(torch.from_numpy(X).cuda())
    exact = torch.zeros_like(fd)
    st, its, _ = p64.solve(lam, fd, exact, rtol=1e-12, maxit=2000)
    assert st == 0
    # correction = exact - c: the step should take it whole
    corr = exact - c
    torch.cuda.synchronize()
    alpha2, rel2 = p.refine(lam, fd, c, corr, r)
    np.testing.assert_allclose(alpha2, 1.0, atol=1e-6)
    assert np.all(rel2 <= 1e-9)
    p.close()
    p64.close()


def _mixed_plans(reqs):
    import torch
    from paper_2402_09531_gb300 import Plan
    plans, fs = [], []
    for r in reqs:
        p = Plan(d=16, kernel="exp", gamma=r.gamma, weight_rule="paper_logrho", q=6.0, eta=2.0, leaf_size=128,
                 precision="mixed", max_rhs=1)
        p.tree_build(torch.from_numpy(r.X).cuda())
        plans.append(p)
        fs.append(torch.from_numpy(r.f).cuda())
    return plans, fs


def test_batched_cg_matches_each_plans_own_cg():
    """dwfmm_batch_cg_step advances the CG of four problems together (one
    fused batch matvec per iteration, fused vector updates): every column
    converges, in about the iterations of the plan's own CG, to the same
    solution within the CG tolerance."""
    import torch
    from paper_2402_09531_gb300 import Batch
    reqs = _requests([1400, 2100, 1000, 2600], seed0=80)
    plans, fs = _mixed_plans(reqs)
    lam, rtol = 1e-1, 1e-6
    single, its1 = [], []
    for p, f in zip(plans, fs):
        p.cg_begin(lam, f, rtol=rtol)
        for _ in range(400):
            p.cg_step(16)
            torch.cuda.synchronize()
            ready, st, it, rr = p.cg_poll()
            if ready and st[0] != 0:
                break
        assert st[0] == 1
        its1.append(int(it[0]))
        c = torch.empty_like(f)
        p.cg_result(c)
        torch.cuda.synchronize()
        single.append(c.cpu().numpy())
    b = Batch(plans, [1] * len(plans))
    for p, f in zip(plans, fs):
        p.cg_begin(lam, f, rtol=rtol)
    for _ in range(400):
        b.cg_step(16)
        torch.cuda.synchronize()
        polls = [p.cg_poll() for p in plans]
        if all(pl[0] and pl[1][0] != 0 for pl in polls):
            break
    for p, f, c1, it1 in zip(plans, fs, single, its1):
        ready, st, it, rr = p.cg_poll()
        assert ready and st[0] == 1
        assert abs(int(it[0]) - it1) <= max(3, it1 // 10)
        c = torch.empty_like(f)
        p.cg_result(c)
        torch.cuda.synchronize()
        c = c.cpu().numpy()
        assert np.linalg.norm(c - c1) / np.linalg.norm(c1) <= 1e-3
    b.close()
    for p in plans:
        p.close()


def test_batched_server_same_within_tolerance_alone_and_in_the_mix():
    """Batched serving (requests of one configuration advance together
    through one batch): every served solve meets rtol with the oracle's
    operator, alone and in the mix, so the two results agree in the
    operator's norm to 2 rtol ||f||."""
    from paper_2402_09531_gb300.serving import Request, Server
    base = _requests([1500, 2600, 900, 3200, 2000, 1200], seed0=90)
    reqs = [Request(rid=r.rid, X=r.X, f=r.f, kernel=r.kernel, gamma=r.gamma, q=r.q, eta=r.eta, leaf=r.leaf,
                    weight_rule=r.weight_rule, lam=1e-2, rtol=1e-6, maxit=4000) for r in base]
    alone = Server(precision="mixed", max_active=1, batched=True)
    r_alone = {r.rid: alone.run([r])[0] for r in reqs[:2]}
    alone.close()
    mix = Server(precision="mixed", max_active=6, batched=True)
    res = {r.rid: r for r in mix.run(reqs)}
    assert mix.peak_active >= 4 and mix.batch_rebuilds >= 2
    mix.close()
    for r in reqs:
        assert res[r.rid].status == "ok", (r.rid, res[r.rid].status)
        assert max(res[r.rid].relres) <= r.rtol
    for rid in (0, 1):
        r = reqs[rid]
        pb = o.make_problem(r.X, "exp", o.weights_paper_normalised(2 * r.gamma, 2.0), 6.0, 128, 2.0)
        A = lambda c: o.fmm_matvec(pb, c[None])[0] + r.lam * c
        fn = np.linalg.norm(r.f[0])
        for c in (res[rid].c[0], r_alone[rid].c[0]):
            assert np.linalg.norm(r.f[0] - A(c)) / fn <= 2e-6
        assert np.linalg.norm(A(res[rid].c[0] - r_alone[rid].c[0])) / fn <= 4e-6


def test_poll_after_a_new_begin_waits_for_its_first_step():
    """A plan reused for a new solve must not report the previous solve's
    status: after dwfmm_cg_begin the poll is not ready until a step ran."""
    import torch
    reqs = _requests([1100], seed0=95)
    plans, fs = _mixed_plans(reqs)
    p, f = plans[0], fs[0]
    p.cg_begin(1e-1, f, rtol=1e-6)
    p.cg_step(8)
    torch.cuda.synchronize()
    assert p.cg_poll()[0]
    p.cg_begin(1e-1, f, rtol=1e-6)
    torch.cuda.synchronize()
    assert not p.cg_poll()[0]
    p.cg_step(4)
    torch.cuda.synchronize()
    ready, st, it, rr = p.cg_poll()
    assert ready and int(it[0]) <= 4
    p.close()


def test_persistent_batch_engine_on_serving_shapes():
    """The persistent batch engine on the serving stream's shape (d = 16,
    exponential kernel, one right-hand side, small problems): bit for bit the
    graph engine's matvec."""
    import torch
    from paper_2402_09531_gb300 import Batch
    reqs = _requests([1400, 2100, 1000, 2600, 1700], seed0=120)
    plans, fs = _mixed_plans(reqs)
    b = Batch(plans, [1] * len(plans))
    out = {}
    for eng in ("graph", "persistent"):
        b.set_engine(eng)
        ys = [torch.full_like(f, float("nan")) for f in fs]
        b.matvec(fs, ys)
        torch.cuda.synchronize()
        out[eng] = ys
    assert b.engine()["persistent_available"]
    for yg, yp in zip(out["graph"], out["persistent"]):
        assert torch.isfinite(yp).all()
        assert torch.equal(yg, yp)
    b.close()
    for p in plans:
        p.close()
