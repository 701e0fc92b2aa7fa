"""Continuous-batching CG solve server on one GPU.

Requests (sites, right-hand sides, kernel parameters) are admitted while an
active slot and enough of the device-memory budget are free.  Every admitted
request owns a plan (from a pool keyed by its expansion parameters, so the
node setup of Sec. 5.4 runs once per configuration), a CUDA stream and its
Krylov state on the device.  Each pass of the loop enqueues a few CG
iterations (dwfmm_cg_step: no host synchronisation) for every request whose
previous batch has finished (dwfmm_cg_poll: never blocks), so the matvecs of
all active requests overlap on the GPU.  A finished inner solve is folded
into the solution with a minimal-residual step against the float64
operator (dwfmm_refine), and float32/mixed plans restart the inner CG on
the float64 residual until it meets the request's tolerance.  Finished requests
release their slot, memory and plan.

With batched=True (float32 / mixed plans) the active requests that share a
configuration (kernel, dimension, weights, index set, leaf size, right-hand
sides) also share one CUDA stream and one batch: every pass advances all of
them with dwfmm_batch_cg_step, whose matvec is one fused launch sequence
over all their problems (their near fields in one launch, their couplings in
another).  The batch is rebuilt whenever a request joins or leaves the group;
each request's Krylov state stays in its own plan, so a rebuild moves
nothing.

This module only schedules; every numerical step runs in libdwfmm.so.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from .dwfmm import Batch, Plan


@dataclass
class Request:
    rid: int
    X: np.ndarray            # (N, d) float64 sites
    f: np.ndarray            # (R, N) float64 right-hand sides
    kernel: str = "exp"
    sigma: float = 1.0
    gamma: np.ndarray | None = None
    q: float = 6.0
    eta: float = 1.0
    leaf: int = 128
    weight_rule: str = "inv_gamma"
    lam: float = 1e-6
    rtol: float = 1e-6
    maxit: int = 5000
    arrival: float = 0.0     # seconds after the start of the run


@dataclass
class Result:
    rid: int
    c: np.ndarray
    status: str              # "ok", "breakdown", "not_converged"
    iters: int
    relres: list
    refinements: int
    t_arrival: float
    t_admit: float
    t_done: float

    @property
    def latency_ms(self) -> float:
        return (self.t_done - self.t_arrival) * 1e3


def estimate_bytes(n: int, d: int, nrhs: int, leaf: int, n_x: int) -> int:
    """Device memory of one request (tree, lists, workspaces, Krylov vectors),
    a deliberately generous upper estimate used for admission."""
    leaves = 2 ** max(0, math.ceil(math.log2(max(1, n) / leaf)))
    clusters = 2 * leaves
    n_pad = (n_x + 7) // 8 * 8
    per_site = d * 8 * 6 + 16 * 4 * 8 + 16 * 8 * 4 + nrhs * 8 * 8 + 64
    per_cluster = n_pad * 16 * 4 * 8 + n_pad * (d + 1) * 12 + d * 8 * 6
    near_pairs = leaves * 64
    # partial sums of the symmetric float64 near field (also run by the
    # float64 residuals of float32 / mixed plans): 2 x upper entries x RHS x leaf
    sym_partials = near_pairs * nrhs * leaf * 8
    return int(n * per_site + clusters * per_cluster + near_pairs * 24 + sym_partials + (32 << 20))


@dataclass
class _Active:
    req: Request
    plan: Plan
    stream: object
    key: tuple
    fd: object               # device rhs of the current inner solve
    f0: object               # device original rhs
    acc: object              # device accumulated solution
    r: object                # device float64 residual f0 - (K64 + lam I) acc
    t_admit: float
    nbytes: int
    iters: int = 0
    refinements: int = 0


@dataclass
class _Group:
    """Requests with one configuration, advanced together (batched mode)."""
    stream: object
    members: list = field(default_factory=list)
    batch: object = None
    dirty: bool = True
    event: object = None      # recorded after the last batched step


class Server:
    """Admission by memory and slots; all active solves advance concurrently."""

    def __init__(self, precision: str = "fp32", max_active: int = 8, mem_budget: int | None = None,
                 step_iters: int = 8, device: int = 0, inner_rtol: float | None = None,
                 inner_maxit: int | None = None, batched: bool = False):
        import torch
        self.torch = torch
        if batched and precision == "fp64":
            raise ValueError("batched serving runs float32 / mixed plans (batches are float32)")
        self.batched = batched
        self.groups: dict = {}        # configuration key -> _Group (batched mode)
        self.batch_rebuilds = 0
        self.dev = torch.device("cuda", device)
        self.precision = precision
        self.max_active = max_active
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            mem_budget = int(0.5 * free)
        self.mem_budget = mem_budget
        self.step_iters = step_iters
        # float32 plans: each inner CG reduces the residual by inner_rtol at most
        # inner_maxit iterations, then the float64 residual restarts it
        # (iterative refinement); float64 plans run one CG to the tolerance.
        self.inner_rtol = inner_rtol if inner_rtol is not None else (1e-3 if precision != "fp64" else None)
        self.inner_maxit = inner_maxit if inner_maxit is not None else (400 if precision != "fp64" else None)
        self.pool: dict = {}
        self.used = 0
        self.peak_active = 0

    # -- plans ----------------------------------------------------------------
    def _key(self, r: Request) -> tuple:
        return (r.X.shape[1], r.kernel, r.sigma, tuple(np.asarray(r.gamma, float)), r.q, r.eta, r.leaf,
                r.weight_rule, r.f.shape[0])

    def _take_plan(self, r: Request, stream) -> tuple:
        key = self._key(r)
        free = self.pool.get(key, [])
        if free:
            return key, free.pop()
        p = Plan(d=r.X.shape[1], kernel=r.kernel, sigma=r.sigma, gamma=r.gamma, weight_rule=r.weight_rule,
                 q=r.q, eta=r.eta, leaf_size=r.leaf, precision=self.precision, max_rhs=r.f.shape[0],
                 stream=stream)
        return key, p

    def _give_plan(self, key, plan: Plan):
        torch = self.torch
        plan.tree_build(torch.zeros((0, plan.d), dtype=torch.float64, device=self.dev))   # release the tree
        self.pool.setdefault(key, []).append(plan)

    # -- request lifecycle ------------------------------------------------------
    def _admit(self, r: Request, t_now: float) -> _Active:
        torch = self.torch
        if self.batched:
            g = self.groups.get(self._key(r))
            if g is None:
                g = self.groups[self._key(r)] = _Group(torch.cuda.Stream(self.dev))
            stream = g.stream
        else:
            stream = torch.cuda.Stream(self.dev)
        key, plan = self._take_plan(r, stream)
        nbytes = estimate_bytes(r.X.shape[0], r.X.shape[1], r.f.shape[0], r.leaf, plan.n_x)
        with torch.cuda.stream(stream):
            Xd = torch.from_numpy(r.X).to(self.dev, non_blocking=False)
            f0 = torch.from_numpy(np.ascontiguousarray(r.f)).to(self.dev)
            acc = torch.zeros_like(f0)
            res = f0.clone()   # the residual of acc = 0
        plan.tree_build(Xd, stream=stream)
        plan.cg_begin(r.lam, f0, rtol=self._inner_tol(r.rtol, 1.0), stream=stream)
        if not self.batched:
            plan.cg_step(self.step_iters, stream=stream)
        self.used += nbytes
        a = _Active(r, plan, stream, key, f0, f0, acc, res, t_now, nbytes)
        if self.batched:
            g = self.groups[key]
            g.members.append(a)
            g.dirty = True
        return a

    def _finish(self, a: _Active, status: str, relres, t_now: float) -> Result:
        torch = self.torch
        a.stream.synchronize()
        c = a.acc.cpu().numpy()
        self.used -= a.nbytes
        self._give_plan(a.key, a.plan)
        return Result(a.req.rid, c, status, a.iters, list(relres), a.refinements, a.req.arrival, a.t_admit, t_now)

    def _inner_tol(self, rtol: float, relres: float) -> float:
        """Relative tolerance of the next inner CG: enough to reach rtol from
        the current float64 relative residual, never tighter than rtol itself,
        and at most inner_rtol for float32 plans."""
        need = max(rtol, 0.5 * rtol / max(relres, 1e-300))
        if self.inner_rtol is not None:
            need = max(need, self.inner_rtol) if relres > rtol / self.inner_rtol else need
        return min(0.5, need)

    def _advance(self, a: _Active, t_now: float):
        """Handle a finished batch of iterations; returns a Result when done."""
        torch = self.torch
        ready, st, its, rr = a.plan.cg_poll()
        if not ready:
            return None
        a_iters = int(its.max()) if len(its) else 0
        running = bool(np.any(st == 0))
        total = a.iters + a_iters
        inner_cap = self.inner_maxit if self.inner_maxit is not None else a.req.maxit
        if running and total < a.req.maxit and a_iters < inner_cap:
            if not self.batched:
                a.plan.cg_step(self.step_iters, stream=a.stream)
            return None
        # inner solve finished: fold its correction in (dwfmm_refine: the plain
        # step where it lowers the float64 residual, else the minimal-residual
        # one, so a poor inner solve cannot raise it)
        with torch.cuda.stream(a.stream):
            delta = torch.empty_like(a.acc)
        a.plan.cg_result(delta, stream=a.stream)
        a.iters = total
        alpha, rel = a.plan.refine(a.req.lam, a.f0, a.acc, delta, a.r, stream=a.stream)
        if np.all(rel <= a.req.rtol):
            return self._finish(a, "ok", rel, t_now)
        if np.any(st == 2) and np.all(alpha == 0.0):
            return self._finish(a, "breakdown", rel, t_now)
        if a.iters >= a.req.maxit or a.refinements >= 60:
            return self._finish(a, "not_converged", rel, t_now)
        # refinement: solve for the float64 residual, relative tolerance rtol of it
        a.refinements += 1
        a.fd = a.r
        a.plan.cg_begin(a.req.lam, a.r, rtol=self._inner_tol(a.req.rtol, float(np.max(rel))), stream=a.stream)
        if not self.batched:
            a.plan.cg_step(self.step_iters, stream=a.stream)
        return None

    def run(self, requests: list) -> list:
        """Serve `requests` (arrival times relative to now); returns results in
        completion order."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list = []
        active: list = []
        done: list = []
        t0 = time.perf_counter()
        pi = 0
        while pi < len(pending) or queue or active:
            now = time.perf_counter() - t0
            while pi < len(pending) and pending[pi].arrival <= now:
                queue.append(pending[pi])
                pi += 1
            while queue and len(active) < self.max_active:
                r = queue[0]
                need = estimate_bytes(r.X.shape[0], r.X.shape[1], r.f.shape[0], r.leaf, 0)
                if active and self.used + need > self.mem_budget:
                    break
                queue.pop(0)
                active.append(self._admit(r, now))
            self.peak_active = max(self.peak_active, len(active))
            progressed = False
            if self.batched:
                progressed = self._step_groups(active, done, t0)
            else:
                for a in list(active):
                    res = self._advance(a, time.perf_counter() - t0)
                    if res is not None:
                        active.remove(a)
                        done.append(res)
                        progressed = True
            if not progressed and not queue:
                time.sleep(20e-6)
        return done

    def _step_groups(self, active: list, done: list, t0: float) -> bool:
        """Batched mode: for every group whose last step has finished, handle
        its members' finished inner solves, rebuild the batch if the
        membership changed, and enqueue the next batched step."""
        torch = self.torch
        progressed = False
        for key, g in list(self.groups.items()):
            if g.event is not None and not g.event.query():
                continue
            for a in list(g.members):
                if g.event is None:
                    break                       # never stepped: nothing to poll yet
                res = self._advance(a, time.perf_counter() - t0)
                if res is not None:
                    g.members.remove(a)
                    active.remove(a)
                    done.append(res)
                    g.dirty = True
                    progressed = True
            if not g.members:
                if g.batch is not None:
                    g.batch.close()
                del self.groups[key]
                continue
            if g.dirty:
                if g.batch is not None:
                    g.batch.close()
                g.batch = Batch([a.plan for a in g.members], [a.req.f.shape[0] for a in g.members],
                                stream=g.stream)
                g.dirty = False
                self.batch_rebuilds += 1
            g.batch.cg_step(self.step_iters, stream=g.stream)
            g.event = torch.cuda.Event()
            g.event.record(g.stream)
        return progressed

    def close(self):
        for g in self.groups.values():
            if g.batch is not None:
                g.batch.close()
        self.groups.clear()
        for plans in self.pool.values():
            for p in plans:
                p.close()
        self.pool.clear()


def summarize(results: list, wall_s: float) -> dict:
    lat = sorted(r.latency_ms for r in results)
    ok = [r for r in results if r.status == "ok"]

    def pct(p):
        if not lat:
            return None
        k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]
    return {"requests": len(results), "ok": len(ok),
            "breakdown": sum(r.status == "breakdown" for r in results),
            "not_converged": sum(r.status == "not_converged" for r in results),
            "p50_ms": pct(50), "p99_ms": pct(99), "solves_per_s": len(results) / wall_s if wall_s > 0 else None,
            "mean_iters": float(np.mean([r.iters for r in results])) if results else None,
            "max_relres": float(max(max(r.relres) for r in ok)) if ok else None}
