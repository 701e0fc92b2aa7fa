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

    python -m paper_2402_09531_gb300.accuracy --n 20000 --r 2 --sigmas 15 --lambdas 3
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


def study(n: int = 20000, d: int = 20, r: float = 2.0, n_sigma: int = 15, n_lambda: int = 15,
          q: float = 8.0, eta: float = 0.5, leaf: int = 128, n_test: int = 1000, n_cols: int = 100,
          repeats: int = 1, seed: int = 0, precision: str = "fp32", maxit: int = 3000,
          lambdas: list | None = None, sigmas: list | None = None) -> dict:
    import torch
    from .dwfmm import Plan

    rng = np.random.default_rng(seed)
    X, b = sample_box(n, d, r, rng)
    X = X - b[None, :] / 2.0                       # the box [-b/2, b/2]: same geometry
    y = target_function(X + b[None, :] / 2.0)
    qx = separation_radius(X)
    diam = float(np.linalg.norm(X.max(0) - X.min(0)))
    if sigmas is None:
        sigmas = list(np.geomspace(max(1e-5, qx), diam, n_sigma))
    if lambdas is None:
        lambdas = list(np.geomspace(1e-6, 1e-1, n_lambda))
    gamma = b / 2.0
    Xd = torch.from_numpy(X).cuda()
    rows = []
    for sigma in sigmas:
        plan = Plan(d=d, kernel="exp", sigma=float(sigma), gamma=gamma, weight_rule="paper_logrho", q=q, eta=eta,
                    leaf_size=leaf, precision=precision, max_rhs=16)
        plan.tree_build(Xd)
        ce = []
        for rep in range(repeats):
            cols = rng.choice(n, size=n_cols, replace=False)
            E = np.zeros((n_cols, n))
            E[np.arange(n_cols), cols] = 1.0
            Kt = np.zeros((n_cols, n))
            for a in range(0, n_cols, 16):
                e = torch.from_numpy(E[a:a + 16].copy()).cuda()
                out = torch.empty_like(e)
                plan.matvec(e, out)
                torch.cuda.synchronize()
                Kt[a:a + 16] = out.cpu().numpy()
            K = np.zeros((n_cols, n))
            for a in range(0, n_cols, 16):
                out = np.zeros((min(16, n_cols - a), n))
                plan.evaluate(X, E[a:a + 16], out)
                K[a:a + 16] = out
            ce.append(float(np.linalg.norm(Kt - K) / np.linalg.norm(K)))
        pe = {}
        for lam in lambdas:
            errs = []
            for rep in range(repeats):
                fd = torch.from_numpy(y[None, :].copy()).cuda()
                cd = torch.zeros_like(fd)
                st, its, rel = plan.solve(float(lam), fd, cd, rtol=1e-6, maxit=maxit)
                T, _ = sample_box(n_test, d, r, rng)
                T = T - b[None, :] / 2.0
                out = np.zeros((1, n_test))
                plan.evaluate(T, cd.cpu().numpy(), out)
                truth = target_function(T + b[None, :] / 2.0)
                errs.append((float(np.linalg.norm(out[0] - truth) / np.linalg.norm(truth)), int(st), int(its)))
            pe[float(lam)] = {"pe": float(np.mean([e[0] for e in errs])), "status": [e[1] for e in errs],
                              "iters": [e[2] for e in errs]}
        rows.append({"sigma": float(sigma), "ce_mean": float(np.mean(ce)), "ce_std": float(np.std(ce)), "pe": pe})
        plan.close()
    return {"n": n, "d": d, "r": r, "q": q, "eta": eta, "q_X": qx, "diam": diam, "rows": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--r", type=float, default=2.0)
    ap.add_argument("--sigmas", type=int, default=15)
    ap.add_argument("--lambdas", type=int, default=3)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--precision", default="fp32")
    args = ap.parse_args()
    res = study(n=args.n, r=args.r, n_sigma=args.sigmas, n_lambda=args.lambdas, repeats=args.repeats,
                precision=args.precision)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
