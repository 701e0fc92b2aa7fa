"""The kernel-interpolation accuracy study of Sec. 6.2, run on the GPU library.

Setup (Sec. 6.2): N uniform samples in [0,1]^20 scaled by b_k = k^-r
(r = 2, 3, 4), exponential kernel exp(-|x-y|/sigma), sigma on a log grid in
[max(1e-5, q_X), diam(B_X)], ridge lambda on a log grid in [1e-6, 1e-1],
eta = 0.5, q = 8 with the normalised weights of Sec. 6.2, CG to a relative
residual of 1e-6, right-hand side y_i = sin(4 pi |x_i|) / (8 pi |x_i|).

* CE (compression error): relative Frobenius error of 100 random columns of
  K_tilde against the same columns of K (K_tilde columns by the matvec on unit
  vectors, K columns by exact evaluation at the sites).
* PE (prediction error): relative 2-norm error of the interpolant at test
  points drawn from the same box, against the function that generated y.

The paper repeats each measurement five times; `repeats` controls that here.
Everything numerical runs in libdwfmm.so (matvec, exact evaluation, CG); this
module draws the inputs and reduces the errors.

    python -m paper_2402_09531_gb300.accuracy --n 100000 --r 2 --ce-only --precision fp64
    python -m paper_2402_09531_gb300.accuracy --n 100000 --r 2 --pe-at 0.0469:1e-6 --precision fp64
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def target_function(X: np.ndarray) -> np.ndarray:
    """y = sin(4 pi |x|) / (8 pi |x|) (Sec. 6.2)."""
    r = np.linalg.norm(X, axis=1)
    r = np.where(r == 0.0, 1e-300, r)
    return np.sin(4.0 * math.pi * r) / (8.0 * math.pi * r)


def sample_box(n: int, d: int, r: float, rng: np.random.Generator) -> np.ndarray:
    b = np.array([float(k) ** (-r) for k in range(1, d + 1)])
    return rng.random((n, d)) * b[None, :], b


def separation_radius(X: np.ndarray) -> float:
    """q_X = min_{i != j} |x_i - x_j| (Def. 2.3), by a k-d tree on the host."""
    from scipy.spatial import cKDTree
    dist, _ = cKDTree(X).query(X, k=2)
    return float(np.min(dist[:, 1]))


def _exact_columns(X: np.ndarray, cols: np.ndarray, sigma: float, precision: str) -> np.ndarray:
    """K[:, cols]^T (len(cols) x N) exactly, by the library's evaluation: a
    plan whose sites are the column sites x_c, evaluated at every site with
    unit coefficients, costs N x len(cols) kernel evaluations."""
    import torch
    from .dwfmm import Plan
    d = X.shape[1]
    m = len(cols)
    sub = Plan(d=d, kernel="exp", sigma=float(sigma), gamma=np.ones(d), q=1.0, eta=1.0,
               leaf_size=max(16, m), precision=precision, max_rhs=16)
    sub.tree_build(np.ascontiguousarray(X[cols]))
    K = np.zeros((m, X.shape[0]))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    for a in range(0, m, 16):
        b = min(m, a + 16)
        E = np.zeros((b - a, m))
        E[np.arange(b - a), np.arange(a, b)] = 1.0
        out = torch.zeros((b - a, X.shape[0]), dtype=torch.float64, device="cuda")
        sub.evaluate(Xd, torch.from_numpy(E).cuda(), out)
        torch.cuda.synchronize()
        K[a:b] = out.cpu().numpy()
    sub.close()
    return K


def compression_error(plan, X: np.ndarray, sigma: float, cols: np.ndarray, precision: str) -> float:
    """CE (Sec. 6.2): relative Frobenius error of the columns `cols` of
    K_tilde (the matvec on unit vectors) against the same columns of K."""
    import torch
    n = X.shape[0]
    Kt = np.zeros((len(cols), n))
    for a in range(0, len(cols), 16):
        b = min(len(cols), a + 16)
        E = np.zeros((b - a, n))
        E[np.arange(b - a), cols[a:b]] = 1.0
        e = torch.from_numpy(E).cuda()
        out = torch.empty_like(e)
        plan.matvec(e, out)
        torch.cuda.synchronize()
        Kt[a:b] = out.cpu().numpy()
    K = _exact_columns(X, cols, sigma, precision)
    return float(np.linalg.norm(Kt - K) / np.linalg.norm(K))


def prediction_error(plan, X: np.ndarray, y: np.ndarray, b: np.ndarray, lam: float, n_test: int,
                     rng: np.random.Generator, maxit: int, rtol: float = 1e-6):
    """PE (Sec. 6.2): solve (K_tilde + lam I) c = y by CG, evaluate the
    interpolant exactly at test points drawn from the box, relative 2-norm
    error against the generating function.  Returns (pe, status, iters)."""
    import torch
    d = X.shape[1]
    fd = torch.from_numpy(y[None, :].copy()).cuda()
    cd = torch.zeros_like(fd)
    st, its, rel = plan.solve(float(lam), fd, cd, rtol=rtol, maxit=maxit)
    T = rng.random((n_test, d)) * b[None, :] - b[None, :] / 2.0
    out = np.zeros((1, n_test))
    plan.evaluate(T, cd.cpu().numpy(), out)
    truth = target_function(T + b[None, :] / 2.0)
    return float(np.linalg.norm(out[0] - truth) / np.linalg.norm(truth)), int(st), int(its)


def problem(n: int, d: int, r: float, seed: int):
    """Sites in the box [-b/2, b/2] (b_k = k^-r; the same geometry as
    [0, b]), the right-hand side at the unshifted points, separation radius
    and diameter."""
    rng = np.random.default_rng(seed)
    X, b = sample_box(n, d, r, rng)
    X = X - b[None, :] / 2.0
    y = target_function(X + b[None, :] / 2.0)
    qx = separation_radius(X)
    diam = float(np.linalg.norm(X.max(0) - X.min(0)))
    return X, y, b, qx, diam, rng


def _plan_for(d, b, sigma, q, eta, leaf, precision):
    from .dwfmm import Plan
    return Plan(d=d, kernel="exp", sigma=float(sigma), gamma=b / 2.0, weight_rule="paper_logrho", q=q, eta=eta,
                leaf_size=leaf, precision=precision, max_rhs=16)


def study(n: int = 20000, d: int = 20, r: float = 2.0, n_sigma: int = 15, n_lambda: int = 15,
          q: float = 8.0, eta: float = 0.5, leaf: int = 128, n_test: int = 1000, n_cols: int = 100,
          repeats: int = 1, seed: int = 0, precision: str = "fp32", maxit: int = 3000,
          lambdas: list | None = None, sigmas: list | None = None, pe: bool = True) -> dict:
    """CE for every sigma of the grid and PE for every (sigma, lambda)."""
    import torch
    X, y, b, qx, diam, rng = problem(n, d, r, seed)
    if sigmas is None:
        sigmas = list(np.geomspace(max(1e-5, qx), diam, n_sigma))
    if lambdas is None:
        lambdas = list(np.geomspace(1e-6, 1e-1, n_lambda))
    Xd = torch.from_numpy(X).cuda()
    rows = []
    for sigma in sigmas:
        plan = _plan_for(d, b, sigma, q, eta, leaf, precision)
        plan.tree_build(Xd)
        ce = [compression_error(plan, X, sigma, rng.choice(n, size=n_cols, replace=False), precision)
              for _ in range(repeats)]
        pes = {}
        for lam in (lambdas if pe else []):
            errs = [prediction_error(plan, X, y, b, lam, n_test, rng, maxit) for _ in range(repeats)]
            pes[float(lam)] = {"pe": float(np.mean([e[0] for e in errs])), "status": [e[1] for e in errs],
                               "iters": [e[2] for e in errs]}
        rows.append({"sigma": float(sigma), "ce_mean": float(np.mean(ce)), "ce_std": float(np.std(ce)),
                     "pe": pes})
        plan.close()
    return {"n": n, "d": d, "r": r, "q": q, "eta": eta, "q_X": qx, "diam": diam, "precision": precision,
            "rows": rows}


def prediction_points(n: int, d: int, r: float, points, q: float = 8.0, eta: float = 0.5, leaf: int = 128,
                      n_test: int = 1000, seed: int = 0, precision: str = "fp64", maxit: int = 20000,
                      repeats: int = 1) -> dict:
    """PE at chosen (sigma, lambda) points (CG to 1e-6)."""
    import torch
    X, y, b, qx, diam, rng = problem(n, d, r, seed)
    Xd = torch.from_numpy(X).cuda()
    out = []
    for sigma, lam in points:
        plan = _plan_for(d, b, sigma, q, eta, leaf, precision)
        plan.tree_build(Xd)
        errs = [prediction_error(plan, X, y, b, lam, n_test, rng, maxit) for _ in range(repeats)]
        out.append({"sigma": float(sigma), "lambda": float(lam), "pe": float(np.mean([e[0] for e in errs])),
                    "pe_std": float(np.std([e[0] for e in errs])), "status": [e[1] for e in errs],
                    "iters": [e[2] for e in errs]})
        plan.close()
    return {"n": n, "d": d, "r": r, "q": q, "eta": eta, "precision": precision, "points": out}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--r", type=float, default=2.0)
    ap.add_argument("--sigmas", type=int, default=15)
    ap.add_argument("--lambdas", type=int, default=3)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--leaf", type=int, default=128)
    ap.add_argument("--maxit", type=int, default=20000)
    ap.add_argument("--ce-only", action="store_true", help="compression error over the sigma grid only")
    ap.add_argument("--pe-at", default=None,
                    help="prediction error at comma-separated sigma:lambda points instead of the grid")
    args = ap.parse_args()
    if args.pe_at:
        pts = [tuple(float(v) for v in p.split(":")) for p in args.pe_at.split(",")]
        res = prediction_points(n=args.n, d=20, r=args.r, points=pts, repeats=args.repeats,
                                precision=args.precision, leaf=args.leaf, maxit=args.maxit)
    else:
        res = study(n=args.n, r=args.r, n_sigma=args.sigmas, n_lambda=args.lambdas, repeats=args.repeats,
                    precision=args.precision, pe=not args.ce_only, leaf=args.leaf, maxit=args.maxit)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
