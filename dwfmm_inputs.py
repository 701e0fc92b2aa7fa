"""Seeded synthetic inputs for the dimension-weighted FMM (DW-FMM).

This module is shared by the FP64 oracle (``oracle/``), the tests and
``bench.py``.  It holds the workload definitions and the random draws only:
none of the method's arithmetic (no weights, no index sets, no kernels).

Workloads follow the paper's synthetic experiments (Sec. 6.2: uniform samples
in an anisotropic box, Sec. 2 Eq. (2.3)): sites are drawn uniformly in the
box prod_k [-gamma_k, gamma_k], right-hand sides are i.i.d. N(0, 1).

Random numbers: NumPy ``default_rng(seed)`` (PCG64).  The sites are drawn
first, as one (N, d) array of U[0, 1) values mapped by x = (2u - 1) * gamma;
the right-hand sides second, as one (R, N) array (R contiguous columns of
length N, i.e. a column-major N x R matrix).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KERNEL_EXP = "exp"            # phi(r) = exp(-r)
KERNEL_MATERN32 = "matern32"  # phi(r) = (1 + sqrt3 r) exp(-sqrt3 r)
KERNEL_GAUSS = "gauss"        # phi(r) = exp(-r^2 / 2)


@dataclass
class Workload:
    """One DW-FMM problem: sites, kernel, index-set degree, tree parameters."""
    name: str
    d: int
    n: int
    gamma: np.ndarray
    kernel: str
    q: float
    leaf: int
    eta: float = 1.0
    nrhs: int = 1
    sigma: float = 1.0
    seed: int = 0
    lam: float = 0.0
    rtol: float = 1e-6
    notes: str = ""
    extra: dict = field(default_factory=dict)


def gamma_inverse_square(d: int) -> np.ndarray:
    """gamma_k = k^-2, k = 1..d."""
    return np.array([1.0 / float(k * k) for k in range(1, d + 1)])


def gamma_sqrt_half(d: int) -> np.ndarray:
    """gamma_k = 2^{-(k-1)/2}, k = 1..d."""
    return np.array([2.0 ** (-(k - 1) / 2.0) for k in range(1, d + 1)])


def gamma_half_powers(d: int) -> np.ndarray:
    """gamma_k = 2^{-k}, k = 1..d."""
    return np.array([2.0 ** (-k) for k in range(1, d + 1)])


def small_exp_d4() -> Workload:
    """d=4, N=4096, gamma=(1,1/2,1/4,1/8), exponential kernel, q=4, leaf 64."""
    return Workload("small_exp_d4_n4096", d=4, n=4096,
                    gamma=np.array([1.0, 0.5, 0.25, 0.125]), kernel=KERNEL_EXP,
                    q=4.0, leaf=64, eta=1.0, nrhs=1, seed=0)


def fp64_matern_d8() -> Workload:
    """d=8, N=262144, gamma_k=k^-2, Matern-3/2, q=6, leaf 128, lambda=1e-6."""
    return Workload("fp64_matern32_d8_n262144", d=8, n=262144,
                    gamma=gamma_inverse_square(8), kernel=KERNEL_MATERN32,
                    q=6.0, leaf=128, eta=1.0, nrhs=1, seed=2, lam=1e-6, rtol=1e-8)


def mixed_gauss_d10() -> Workload:
    """d=10, N=2^20, gamma_k=2^{-(k-1)/2}, Gaussian, q=8, leaf 256, 16 RHS."""
    return Workload("mixed_gauss_d10_n1048576_r16", d=10, n=1048576,
                    gamma=gamma_sqrt_half(10), kernel=KERNEL_GAUSS,
                    q=8.0, leaf=256, eta=1.0, nrhs=16, seed=3, lam=1e-6, rtol=1e-6)


def scaled(w: Workload, n: int, nrhs: int | None = None, name: str | None = None) -> Workload:
    """Same workload shape at another N (and optionally another RHS count)."""
    return Workload(name or f"{w.name}@N{n}", d=w.d, n=n, gamma=w.gamma.copy(),
                    kernel=w.kernel, q=w.q, leaf=w.leaf, eta=w.eta,
                    nrhs=w.nrhs if nrhs is None else nrhs, sigma=w.sigma,
                    seed=w.seed, lam=w.lam, rtol=w.rtol)


def sites(w: Workload) -> np.ndarray:
    """(N, d) float64 sites uniform in prod_k [-gamma_k, gamma_k] (drawn first)."""
    rng = np.random.default_rng(w.seed)
    u = rng.random((w.n, w.d))
    return (2.0 * u - 1.0) * w.gamma[None, :]


def sites_and_rhs(w: Workload, nrhs: int | None = None):
    """Sites (N, d) then right-hand sides (R, N), both from one seeded stream."""
    rng = np.random.default_rng(w.seed)
    u = rng.random((w.n, w.d))
    x = (2.0 * u - 1.0) * w.gamma[None, :]
    r = w.nrhs if nrhs is None else nrhs
    f = rng.standard_normal((r, w.n))
    return x, f


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """(R, N) standard normal right-hand sides from their own seed."""
    return np.random.default_rng(seed).standard_normal((nrhs, n))


def batching_problems(count: int = 256, seed: int = 4):
    """Many uneven problems: N log-uniform in [2048, 65536], d in {6..12},
    gamma_k = k^-2, Matern-3/2, q = 5, 1-8 right-hand sides each."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(round(math.exp(rng.uniform(math.log(2048), math.log(65536)))))
        d = int(rng.integers(6, 13))
        r = int(rng.integers(1, 9))
        out.append(Workload(f"batch{p}", d=d, n=n, gamma=gamma_inverse_square(d),
                            kernel=KERNEL_MATERN32, q=5.0, leaf=128, eta=1.0,
                            nrhs=r, seed=seed * 100003 + p))
    return out


def serving_requests(count: int = 2000, seed: int = 5, nmin: float = 1e3, nmax: float = 5e5):
    """CG solve requests: N log-uniform in [nmin, nmax], d=16, gamma_k=2^-k,
    exponential kernel, q=6, lambda=1e-6, rtol=1e-6."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        out.append(Workload(f"req{p}", d=16, n=n, gamma=gamma_half_powers(16),
                            kernel=KERNEL_EXP, q=6.0, leaf=128, eta=1.0, nrhs=1,
                            seed=seed * 100003 + p, lam=1e-6, rtol=1e-6))
    return out
