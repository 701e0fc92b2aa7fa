"""Plain FP64 CPU oracle of the dimension-weighted fast multipole method.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
statement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The library in ``paper_2402_09531_gb300/``
never imports it, and the two share no code: only the seeded input
generators of ``dwfmm_inputs`` serve both.

Harbrecht, Multerer, Quizi, "The dimension weighted fast multipole method for
scattered data approximation" (arXiv 2402.09531).  Every function cites the
section / equation it follows.  Where the paper is silent or garbled, the
reading taken here is stated in the docstring (tagged "Reading").

Everything is float64.  No blocking, fusion or reordering beyond what the
definitions state; loops run in the paper's order.  Library primitives used
as single steps: numpy matmul, numpy.linalg.solve, argsort.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, invariants or brute force.  The
printed count 244 of Sec. 6.1 is not reproduced by any reading of the weight
rule tried here; that single number is "parity unpinned" (the structural
claims of Sec. 6.1 are pinned instead).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Kernels (Sec. 2; Sec. 6.2 / 6.3 use the exponential kernel).
# Reading: Sec. 6.2 prints exp(+|x-y|/sigma); only exp(-|x-y|/sigma) is
# positive definite (Def. 2.2), so the minus sign is used.
# ---------------------------------------------------------------------------

def kernel_phi(kind: str, r, sigma: float = 1.0):
    """phi(r / sigma) for the three radial kernels used by the workloads."""
    s = np.asarray(r, dtype=np.float64) / sigma
    if kind == "exp":
        return np.exp(-s)
    if kind == "matern32":
        t = math.sqrt(3.0) * s
        return (1.0 + t) * np.exp(-t)
    if kind == "gauss":
        return np.exp(-0.5 * s * s)
    raise ValueError(f"unknown kernel {kind!r}")


def kernel_matrix(kind: str, X: np.ndarray, Y: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """[K(x_i, y_j)]_{i,j} with Euclidean distance (Sec. 2, matrix K)."""
    diff = X[:, None, :] - Y[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    return kernel_phi(kind, r, sigma)


# ---------------------------------------------------------------------------
# Weights (Lemma 4.1, Theorem 4.6, Sec. 6.2)
# ---------------------------------------------------------------------------

def rho_of_tau(tau):
    """rho = 2 tau + sqrt(1 + 4 tau^2) (Lemma 4.1)."""
    tau = np.asarray(tau, dtype=np.float64)
    return 2.0 * tau + np.sqrt(1.0 + 4.0 * tau * tau)


def weights_log_rho(tau) -> np.ndarray:
    """omega_k = log rho_k (Theorem 4.6)."""
    return np.log(rho_of_tau(tau))


def weights_paper_normalised(b, eta: float) -> np.ndarray:
    """Sec. 6.2: tau_k^{-1} = eta b_k, rho_k = e rho(tau_k) / rho(tau_1),
    omega_k = log rho_k, so that omega_1 = 1."""
    b = np.asarray(b, dtype=np.float64)
    tau = 1.0 / (eta * b)
    rho = math.e * rho_of_tau(tau) / rho_of_tau(tau[0])
    return np.log(rho)


def weights_inv_gamma(gamma) -> np.ndarray:
    """Reading for the workloads: omega_k = gamma_1 / gamma_k (equal to the
    literal 1/gamma_k whenever gamma_1 = 1; normalised to omega_1 = 1 as in
    Sec. 6.2 otherwise)."""
    g = [float(v) for v in gamma]
    return np.array([g[0] / gk for gk in g])


# ---------------------------------------------------------------------------
# Weighted total-degree index set (Sec. 4, Lambda_{omega,q,d})
# ---------------------------------------------------------------------------

def index_set(w, q: float, shape: str = "total") -> np.ndarray:
    """All alpha in N^d with sum_l omega_l alpha_l <= q (Sec. 4), or, for
    shape "tensor", with max_l omega_l alpha_l <= q (the tensor-product set
    ||alpha||_inf <= q of Sec. 6.1 when omega = 1).

    Reading: the comparison is inclusive with a relative slack of 1e-12
    (sum <= q (1 + 1e-12)); the sum is accumulated left to right in float64
    (s_k = s_{k-1} + omega_k alpha_k).  Enumeration order: lexicographic in
    (alpha_1, ..., alpha_d), alpha_1 most significant.
    """
    if shape == "tensor":
        w = [float(v) for v in w]
        if any(not (v > 0.0) for v in w):
            raise ValueError("weights must be positive")
        tol = float(q) * (1.0 + 1e-12)
        ranges = []
        for v in w:                       # the a >= 0 with omega_k a <= q, one by one
            a = 0
            while v * float(a + 1) <= tol:
                a += 1
            ranges.append(range(a + 1))
        # itertools.product varies the last index fastest: lexicographic order
        out = [list(a) for a in itertools.product(*ranges)]
        return np.array(out, dtype=np.int64).reshape(len(out), len(w))
    if shape != "total":
        raise ValueError("shape must be 'total' or 'tensor'")
    w = [float(v) for v in w]
    d = len(w)
    if any(not (v > 0.0) for v in w):
        raise ValueError("weights must be positive")
    tol = float(q) * (1.0 + 1e-12)
    out = []
    alpha = [0] * d

    def rec(k: int, s: float):
        if k == d:
            out.append(list(alpha))
            return
        a = 0
        while True:
            t = s + w[k] * float(a)
            if t > tol:
                break
            alpha[k] = a
            rec(k + 1, t)
            a += 1
        alpha[k] = 0

    rec(0, 0.0)
    return np.array(out, dtype=np.int64).reshape(len(out), d)


def tensor_index_count(q: int, d: int) -> int:
    """|{alpha : ||alpha||_inf <= q}| = (q+1)^d (Sec. 6.1), in exact integers."""
    return math.prod([q + 1] * d)


# ---------------------------------------------------------------------------
# Orthonormal Legendre basis on [0, 1] (Sec. 5.2)
# ---------------------------------------------------------------------------

def legendre_hat(jmax: int, t) -> np.ndarray:
    """p_hat_j(t) = sqrt(2j+1) P_j(2t - 1), j = 0..jmax, orthonormal on [0,1].

    P_j by the three-term recurrence (j+1) P_{j+1} = (2j+1) u P_j - j P_{j-1}.
    Returns an array of shape (jmax + 1, len(t)).
    """
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    u = 2.0 * t - 1.0
    P = np.zeros((jmax + 1, t.size))
    P[0] = 1.0
    if jmax >= 1:
        P[1] = u
    for j in range(1, jmax):
        P[j + 1] = ((2 * j + 1) * u * P[j] - j * P[j - 1]) / (j + 1)
    scale = np.sqrt(2.0 * np.arange(jmax + 1) + 1.0)
    return P * scale[:, None]


def basis_eval(Lam: np.ndarray, T: np.ndarray) -> np.ndarray:
    """[p_hat_alpha(t)]_{t in T, alpha in Lambda}: tensor Legendre (Sec. 5.2).

    T has shape (npts, d) in [0,1]^d; returns (npts, n)."""
    T = np.atleast_2d(np.asarray(T, dtype=np.float64))
    npts, d = T.shape
    out = np.ones((npts, Lam.shape[0]))
    for k in range(d):
        jmax = int(Lam[:, k].max()) if Lam.shape[0] else 0
        Pk = legendre_hat(jmax, T[:, k])          # (jmax+1, npts)
        out *= Pk[Lam[:, k], :].T
    return out


# ---------------------------------------------------------------------------
# Halton candidates and approximate Fekete points (Sec. 5.4)
# ---------------------------------------------------------------------------

def first_primes(d: int) -> list[int]:
    """The first d primes (bases of the Halton sequence)."""
    out, c = [], 2
    while len(out) < d:
        if all(c % p for p in out if p * p <= c):
            out.append(c)
        c += 1
    return out


def radical_inverse(i: int, base: int) -> float:
    """Digit-reversed fraction of i in the given base (Halton's definition).

    Reading: computed as one integer ratio R / base^k (k = number of digits),
    i.e. the correctly rounded value of the exact radical inverse."""
    num, den = 0, 1
    while i > 0:
        i, digit = divmod(i, base)
        num = num * base + digit
        den *= base
    return num / den


def halton(M: int, d: int, start: int = 1) -> np.ndarray:
    """Halton points h_i, i = start..start+M-1, coordinate k in base prime_k.

    Reading (unstated in Sec. 5.4): first d primes, start at i = 1 (the origin
    is skipped), no scrambling."""
    pr = first_primes(d)
    H = np.empty((M, d))
    for r in range(M):
        for k in range(d):
            H[r, k] = radical_inverse(start + r, pr[k])
    return H


def halton_count(n: int) -> int:
    """Reading: number of Halton candidates M = max(2000, 10 n)."""
    return max(2000, 10 * n)


def greedy_cpqr(A: np.ndarray) -> list[int]:
    """Column-pivoted QR on A (rows: polynomials, columns: candidates), greedy.

    Sec. 5.4: approximate Fekete points are the columns picked by a QR
    decomposition with column pivoting of the Vandermonde matrix on the
    candidates.  At each step the column with the largest remaining 2-norm
    is picked (ties: lowest index), normalised, and projected out of every
    column (modified Gram-Schmidt); norms are recomputed, not downdated.
    Returns the n picked column indices in pick order.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    n, M = R.shape
    if M < n:
        raise ValueError("fewer candidates than polynomials")
    picked: list[int] = []
    alive = np.ones(M, dtype=bool)
    for _ in range(n):
        norms2 = np.sum(R * R, axis=0)
        norms2[~alive] = -1.0
        p = int(np.argmax(norms2))
        if not norms2[p] > 0.0:
            raise np.linalg.LinAlgError("candidates are not unisolvent")
        picked.append(p)
        alive[p] = False
        qv = R[:, p] / math.sqrt(norms2[p])
        R -= np.outer(qv, qv @ R)
    return picked


@dataclass
class Expansion:
    """Far-field expansion data shared by all clusters (Sec. 4, 5.2, 5.4)."""
    weights: np.ndarray   # omega, (d,)
    Lam: np.ndarray       # Lambda, (n, d)
    nodes: np.ndarray     # xi_hat, (n, d) in [0,1]^d, row s = s-th pivot
    pivots: list          # candidate indices of the nodes
    V: np.ndarray         # [p_hat_alpha'(xi_hat_alpha)], (n, n)

    @property
    def n(self) -> int:
        return self.Lam.shape[0]


def make_expansion(weights, q: float, nodes: np.ndarray | None = None,
                   M: int | None = None, shape: str = "total") -> Expansion:
    """Index set, approximate Fekete nodes and Vandermonde matrix (Eq. (5.3))."""
    Lam = index_set(weights, q, shape)
    n, d = Lam.shape
    pivots: list = []
    if nodes is None:
        M = halton_count(n) if M is None else M
        H = halton(M, d)
        A = basis_eval(Lam, H).T                  # (n, M)
        pivots = greedy_cpqr(A)
        nodes = H[pivots]
    nodes = np.asarray(nodes, dtype=np.float64)
    V = basis_eval(Lam, nodes)                    # V[s, alpha'] = p_hat_alpha'(xi_s)
    return Expansion(np.asarray(weights, dtype=np.float64), Lam, nodes, pivots, V)


# ---------------------------------------------------------------------------
# Cluster tree (Sec. 5.1, Def. 5.1 and 5.2)
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    """Balanced binary cluster tree, clusters numbered level-wise:
    level j holds clusters 2^j - 1 .. 2^{j+1} - 2 (heap order)."""
    n: int
    d: int
    depth: int            # J
    perm: np.ndarray      # tree position -> original site index
    begin: np.ndarray     # per cluster, into tree order
    end: np.ndarray
    lo: np.ndarray        # tight bounding box, (clusters, d)
    hi: np.ndarray

    def level_range(self, j: int):
        return (1 << j) - 1, (1 << (j + 1)) - 1

    @property
    def nclusters(self) -> int:
        return (1 << (self.depth + 1)) - 1


def tree_depth(n: int, leaf: int) -> int:
    """Reading: J = smallest integer with ceil(n / 2^J) <= leaf, so every
    leaf has at most `leaf` sites and all leaves sit on level J (Def. 5.2)."""
    J = 0
    while -(-n // (1 << J)) > leaf:
        J += 1
    return J


def bounding_box(P: np.ndarray):
    """Smallest axis-parallel cuboid holding the rows of P (Def. 5.1)."""
    return P.min(axis=0), P.max(axis=0)


def build_tree(X: np.ndarray, leaf: int) -> Tree:
    """Cardinality-balanced clustering (Sec. 5.1).

    Each cluster at level j < J is split along the longest edge of its
    bounding box (ties: lowest k) so that both halves hold (nearly) the same
    number of sites.  Reading: the first child takes the ceil(n/2) sites that
    are smallest by (x_k, current position); both children keep the parent's
    relative order (stable partition).
    """
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    if leaf < 2:
        raise ValueError("leaf size must be >= 2")
    J = tree_depth(n, leaf) if n > 0 else 0
    nc = (1 << (J + 1)) - 1
    perm = np.arange(n)
    begin = np.zeros(nc, dtype=np.int64)
    end = np.zeros(nc, dtype=np.int64)
    begin[0], end[0] = 0, n
    for j in range(J):
        first, last = (1 << j) - 1, (1 << (j + 1)) - 1
        for c in range(first, last):
            b, e = int(begin[c]), int(end[c])
            idx = perm[b:e].copy()
            P = X[idx]
            lo, hi = bounding_box(P)
            k = int(np.argmax(hi - lo))
            n1 = -(-(e - b) // 2)
            order = np.lexsort((np.arange(e - b), P[:, k]))   # by x_k, then position
            left = np.zeros(e - b, dtype=bool)
            left[order[:n1]] = True
            perm[b:e] = np.concatenate([idx[left], idx[~left]])
            c1, c2 = 2 * c + 1, 2 * c + 2
            begin[c1], end[c1] = b, b + n1
            begin[c2], end[c2] = b + n1, e
    lo = np.zeros((nc, d))
    hi = np.zeros((nc, d))
    for c in range(nc):
        b, e = int(begin[c]), int(end[c])
        if e > b:
            lo[c], hi[c] = bounding_box(X[perm[b:e]])
    return Tree(n, d, J, perm, begin, end, lo, hi)


def affine_extent(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Edge lengths of the affine map a_nu: [0,1]^d -> B_nu (Sec. 5.2).

    Reading: a degenerate edge (zero length) is widened to
    1e-12 * max(1, longest edge) so that a_nu stays invertible."""
    ext = hi - lo
    guard = 1e-12 * max(1.0, float(np.max(ext)) if ext.size else 1.0)
    return np.maximum(ext, guard)


def to_reference(lo, ext, P):
    """a_nu^{-1}(x) = (x - lo) / ext (Sec. 5.2)."""
    return (P - lo[None, :]) / ext[None, :]


def from_reference(lo, ext, T):
    """a_nu(t) = lo + t * ext (Sec. 5.2)."""
    return lo[None, :] + T * ext[None, :]


# ---------------------------------------------------------------------------
# Admissibility and far/near lists (Sec. 5.2, Eq. (5.1))
# ---------------------------------------------------------------------------

def admissible(lo1, hi1, lo2, hi2, eta: float) -> bool:
    """dist(B, B') >= eta * max(diam B, diam B') (Eq. (5.1)).

    Reading: compared in squares, sums accumulated over k in order, each
    term a product then an add (no fused multiply-add).  A pair at distance
    zero is never admissible (this only matters for single-site clusters)."""
    D2 = 0.0
    da = 0.0
    db = 0.0
    for k in range(len(lo1)):
        g = max(0.0, float(lo2[k]) - float(hi1[k]), float(lo1[k]) - float(hi2[k]))
        D2 = D2 + g * g
        ea = float(hi1[k]) - float(lo1[k])
        eb = float(hi2[k]) - float(lo2[k])
        da = da + ea * ea
        db = db + eb * eb
    return D2 > 0.0 and D2 >= (eta * eta) * max(da, db)


@dataclass
class Lists:
    """far[j]: admissible same-level pairs (t, s) at level j whose parents are
    not admissible; near: non-admissible leaf pairs.  Both sorted by (t, s)."""
    far: list
    near: np.ndarray


def admissible_pairs(lo: np.ndarray, hi: np.ndarray, t: np.ndarray, s: np.ndarray,
                     eta: float) -> np.ndarray:
    """Eq. (5.1) for many pairs at once, with the same float64 operations in
    the same order as `admissible` (products and adds over k, no fused
    multiply-add), so both give identical decisions."""
    D2 = np.zeros(t.size)
    da = np.zeros(t.size)
    db = np.zeros(t.size)
    for k in range(lo.shape[1]):
        g = np.maximum(0.0, np.maximum(lo[s, k] - hi[t, k], lo[t, k] - hi[s, k]))
        D2 = D2 + g * g
        ea = hi[t, k] - lo[t, k]
        eb = hi[s, k] - lo[s, k]
        da = da + ea * ea
        db = db + eb * eb
    return (D2 > 0.0) & (D2 >= (eta * eta) * np.maximum(da, db))


def build_lists(tree: Tree, eta: float) -> Lists:
    """Level-wise block-cluster tree traversal (Sec. 5.2).

    Reading of the garbled farfield definition: nu x nu' is in F iff it is
    admissible and parent(nu) x parent(nu') is not; N holds the leaf pairs
    that are not admissible.  Both orderings (nu, nu') and (nu', nu) are kept.
    Candidates of one level are tested together (`admissible_pairs`).
    """
    J = tree.depth
    far = [np.zeros((0, 2), dtype=np.int64) for _ in range(J + 1)]
    near = np.zeros((0, 2), dtype=np.int64)
    if tree.n == 0:
        return Lists(far, near)
    ct = np.array([0], dtype=np.int64)
    cs = np.array([0], dtype=np.int64)
    for j in range(J + 1):
        order = np.lexsort((cs, ct))
        ct, cs = ct[order], cs[order]
        adm = admissible_pairs(tree.lo, tree.hi, ct, cs, eta)
        far[j] = np.stack([ct[adm], cs[adm]], axis=1)
        nt, ns = ct[~adm], cs[~adm]
        if j == J:
            near = np.stack([nt, ns], axis=1)
            break
        ct = np.concatenate([2 * nt + a for a in (1, 2) for b in (1, 2)])
        cs = np.concatenate([2 * ns + b for a in (1, 2) for b in (1, 2)])
    return Lists(far, near)


# ---------------------------------------------------------------------------
# Cluster bases, transfer and coupling matrices (Sec. 5.2, Eq. (5.2)-(5.4))
# ---------------------------------------------------------------------------

def cluster_basis(exp_: Expansion, tree: Tree, c: int, X: np.ndarray) -> np.ndarray:
    """P_nu = [p^nu_alpha(x)]_{x in nu, alpha} with p^nu = p_hat o a_nu^{-1}."""
    b, e = int(tree.begin[c]), int(tree.end[c])
    ext = affine_extent(tree.lo[c], tree.hi[c])
    T = to_reference(tree.lo[c], ext, X[tree.perm[b:e]])
    return basis_eval(exp_.Lam, T)


def transfer_matrix(exp_: Expansion, tree: Tree, child: int) -> np.ndarray:
    """T_child = V^{-1} [p^nu_alpha'(a_child(xi_hat_alpha))]_{alpha,alpha'},
    nu = parent(child) (Sec. 5.2, two-scale relation)."""
    parent = (child - 1) // 2
    ec = affine_extent(tree.lo[child], tree.hi[child])
    ep = affine_extent(tree.lo[parent], tree.hi[parent])
    Y = from_reference(tree.lo[child], ec, exp_.nodes)          # a_child(xi)
    Bm = basis_eval(exp_.Lam, to_reference(tree.lo[parent], ep, Y))
    return np.linalg.solve(exp_.V, Bm)


def coupling_matrix(exp_: Expansion, tree: Tree, t: int, s: int, kernel: str,
                    sigma: float) -> np.ndarray:
    """S_{nu,nu'} = [K(a_nu(xi_alpha), a_nu'(xi_alpha'))] (Sec. 5.2)."""
    Yt = from_reference(tree.lo[t], affine_extent(tree.lo[t], tree.hi[t]), exp_.nodes)
    Ys = from_reference(tree.lo[s], affine_extent(tree.lo[s], tree.hi[s]), exp_.nodes)
    return kernel_matrix(kernel, Yt, Ys, sigma)


def coefficient_matrix(exp_: Expansion, S: np.ndarray) -> np.ndarray:
    """C_{nu,nu'} = V^{-1} S_{nu,nu'} V^{-T} (Sec. 5.2)."""
    W = np.linalg.solve(exp_.V, S)                 # V^{-1} S
    return np.linalg.solve(exp_.V, W.T).T          # (V^{-1} (V^{-1} S)^T)^T


# ---------------------------------------------------------------------------
# The DW-FMM matrix-vector product (Eq. (5.4) with nested bases)
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """Sites, kernel and the structures the FMM needs.  `cache` memoizes the
    matrices that depend on the tree only (T_c and C_{t,s}), so repeated
    matvecs on one tree do not recompute them; the arithmetic is unchanged."""
    X: np.ndarray
    kernel: str
    sigma: float
    exp_: Expansion
    tree: Tree
    lists: Lists
    cache: dict = field(default_factory=dict)


def problem_transfer(pb: Problem, c: int) -> np.ndarray:
    """T_c of Sec. 5.2 for this problem's tree (memoized)."""
    key = ("T", c)
    if key not in pb.cache:
        pb.cache[key] = transfer_matrix(pb.exp_, pb.tree, c)
    return pb.cache[key]


def problem_coefficient(pb: Problem, t: int, s: int) -> np.ndarray:
    """C_{t,s} = V^{-1} S_{t,s} V^{-T} for this problem's tree (memoized)."""
    key = ("C", t, s)
    if key not in pb.cache:
        S = coupling_matrix(pb.exp_, pb.tree, t, s, pb.kernel, pb.sigma)
        pb.cache[key] = coefficient_matrix(pb.exp_, S)
    return pb.cache[key]


def make_problem(X, kernel: str, weights, q: float, leaf: int, eta: float,
                 sigma: float = 1.0, nodes=None, shape: str = "total") -> Problem:
    X = np.asarray(X, dtype=np.float64)
    exp_ = make_expansion(weights, q, nodes=nodes, shape=shape)
    tree = build_tree(X, leaf)
    lists = build_lists(tree, eta)
    return Problem(X, kernel, sigma, exp_, tree, lists)


def upward_pass(pb: Problem, xt: np.ndarray) -> dict:
    """Moments mu_nu = P_nu^T x_nu, computed at the leaves and carried up by
    the two-scale relation mu_nu = sum_c T_c^T mu_c (Sec. 5.2).
    xt: (N, R) right-hand sides in tree order."""
    tr = pb.tree
    J = tr.depth
    mu = {}
    f, l = tr.level_range(J)
    for c in range(f, l):
        b, e = int(tr.begin[c]), int(tr.end[c])
        mu[c] = cluster_basis(pb.exp_, tr, c, pb.X).T @ xt[b:e]
    for j in range(J - 1, -1, -1):
        f, l = tr.level_range(j)
        for c in range(f, l):
            acc = 0.0
            for ch in (2 * c + 1, 2 * c + 2):
                acc = acc + problem_transfer(pb, ch).T @ mu[ch]
            mu[c] = acc
    return mu


def farfield_coefficients(pb: Problem, mu: dict, targets=None) -> dict:
    """lambda_nu = sum_{nu' : (nu,nu') in F} C_{nu,nu'} mu_nu' (Eq. (5.4)).
    If `targets` is given, only those target clusters are computed."""
    lam = {}
    for j, pairs in enumerate(pb.lists.far):
        for (t, s) in pairs:
            t, s = int(t), int(s)
            if targets is not None and t not in targets:
                continue
            lam[t] = lam.get(t, 0.0) + problem_coefficient(pb, t, s) @ mu[s]
    return lam


def downward_pass(pb: Problem, lam: dict, R: int, leaves=None) -> dict:
    """lambda_c += T_c lambda_parent(c) from the root to the leaves (Sec. 5.2).
    Returns the accumulated coefficients of the leaves (or of `leaves`)."""
    tr = pb.tree
    n = pb.exp_.n
    acc = {}
    need = None
    if leaves is not None:
        need = set()
        for c in leaves:
            while True:
                need.add(c)
                if c == 0:
                    break
                c = (c - 1) // 2
    for j in range(tr.depth + 1):
        f, l = tr.level_range(j)
        for c in range(f, l):
            if need is not None and c not in need:
                continue
            v = np.zeros((n, R)) + lam.get(c, 0.0)
            if c > 0:
                v = v + problem_transfer(pb, c) @ acc[(c - 1) // 2]
            acc[c] = v
    f, l = tr.level_range(tr.depth)
    return {c: acc[c] for c in range(f, l) if c in acc}


def nearfield(pb: Problem, xt: np.ndarray, t: int) -> np.ndarray:
    """sum over (t, s) in N of K_{t,s} x_s (dense near-field blocks)."""
    tr = pb.tree
    b, e = int(tr.begin[t]), int(tr.end[t])
    out = np.zeros((e - b, xt.shape[1]))
    rows = pb.lists.near[pb.lists.near[:, 0] == t] if pb.lists.near.size else []
    Xt = pb.X[tr.perm[b:e]]
    for (_, s) in rows:
        bs, es = int(tr.begin[s]), int(tr.end[s])
        K = kernel_matrix(pb.kernel, Xt, pb.X[tr.perm[bs:es]], pb.sigma)
        out += K @ xt[bs:es]
    return out


def fmm_matvec(pb: Problem, x: np.ndarray) -> np.ndarray:
    """y = K_tilde x (Eq. (5.4), nested bases); x and y are (R, N) in the
    caller's site order."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    R, N = x.shape
    tr = pb.tree
    if N == 0:
        return np.zeros((R, 0))
    xt = x[:, tr.perm].T                          # (N, R) tree order
    mu = upward_pass(pb, xt)
    lam = farfield_coefficients(pb, mu)
    loc = downward_pass(pb, lam, R)
    yt = np.zeros((N, R))
    f, l = tr.level_range(tr.depth)
    for c in range(f, l):
        b, e = int(tr.begin[c]), int(tr.end[c])
        yt[b:e] = cluster_basis(pb.exp_, tr, c, pb.X) @ loc[c] + nearfield(pb, xt, c)
    y = np.empty((R, N))
    y[:, tr.perm] = yt.T
    return y


def fmm_matvec_leaves(pb: Problem, x: np.ndarray, leaves) -> dict:
    """Rows of y = K_tilde x for the target leaves in `leaves` only.

    Full upward pass; far-field coefficients only for the leaves' ancestors;
    downward pass along those chains; leaf evaluation plus near field.
    Returns {leaf: (|leaf|, R) array in tree order within the leaf}."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    R, N = x.shape
    tr = pb.tree
    xt = x[:, tr.perm].T
    mu = upward_pass(pb, xt)
    anc = set()
    for c in leaves:
        while True:
            anc.add(int(c))
            if c == 0:
                break
            c = (c - 1) // 2
    lam = farfield_coefficients(pb, mu, targets=anc)
    loc = downward_pass(pb, lam, R, leaves=[int(c) for c in leaves])
    out = {}
    for c in leaves:
        c = int(c)
        out[c] = cluster_basis(pb.exp_, tr, c, pb.X) @ loc[c] + nearfield(pb, xt, c)
    return out


def assemble_ktilde(pb: Problem) -> np.ndarray:
    """Explicit K_tilde (tiny N only), in the caller's order.

    Far blocks use each block's own cluster bases directly,
    K_tilde_{nu,nu'} = P_nu V^{-1} S V^{-T} P_nu'^T (Eq. (5.4)), not the
    nested transfers; near blocks are K_{nu,nu'}."""
    tr = pb.tree
    N = tr.n
    Kt = np.zeros((N, N))
    for pairs in pb.lists.far:
        for (t, s) in pairs:
            t, s = int(t), int(s)
            Pt = cluster_basis(pb.exp_, tr, t, pb.X)
            Ps = cluster_basis(pb.exp_, tr, s, pb.X)
            S = coupling_matrix(pb.exp_, tr, t, s, pb.kernel, pb.sigma)
            C = coefficient_matrix(pb.exp_, S)
            bt, et = int(tr.begin[t]), int(tr.end[t])
            bs, es = int(tr.begin[s]), int(tr.end[s])
            Kt[bt:et, bs:es] = Pt @ C @ Ps.T
    for (t, s) in pb.lists.near:
        t, s = int(t), int(s)
        bt, et = int(tr.begin[t]), int(tr.end[t])
        bs, es = int(tr.begin[s]), int(tr.end[s])
        Kt[bt:et, bs:es] = kernel_matrix(pb.kernel, pb.X[tr.perm[bt:et]],
                                         pb.X[tr.perm[bs:es]], pb.sigma)
    out = np.empty_like(Kt)
    out[np.ix_(tr.perm, tr.perm)] = Kt
    return out


def dense_matvec(kind: str, X: np.ndarray, x: np.ndarray, sigma: float = 1.0,
                 rows=None, chunk: int = 2048) -> np.ndarray:
    """Brute force y = K x (Sec. 2), optionally only for the sites in `rows`.
    x: (R, N); returns (R, len(rows)) or (R, N)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    idx = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    y = np.zeros((x.shape[0], idx.size))
    for a in range(0, idx.size, chunk):
        sl = idx[a:a + chunk]
        for b in range(0, X.shape[0], 8192):
            K = kernel_matrix(kind, X[sl], X[b:b + 8192], sigma)
            y[:, a:a + sl.size] += (K @ x[:, b:b + 8192].T).T
    return y


# ---------------------------------------------------------------------------
# Conjugate gradients for (K_tilde + lambda I) c = f (Sec. 2 Eq. (2.2), Sec. 6.2)
# ---------------------------------------------------------------------------

@dataclass
class CGResult:
    c: np.ndarray
    iters: int
    relres: float
    status: str     # "ok", "breakdown", "not_converged"


def cg(apply, f: np.ndarray, lam: float, rtol: float, maxit: int) -> CGResult:
    """Unpreconditioned Hestenes-Stiefel CG with x0 = 0 on v -> A v + lam v.

    Reading (Sec. 6.2 "relative error less than 1e-6"): stop when the
    recurrence residual satisfies ||r_k|| <= rtol ||f||; the reported relres
    is the true residual ||f - (A + lam I) c|| / ||f||.  Sec. 6.2 runs CG on
    the compressed matrix with ridges down to 1e-6, and the compression error
    (Sec. 5.3) can make K_tilde + lam I mildly indefinite, so negative
    curvature p^T A p < 0 does not stop the iteration; breakdown is only
    p^T A p == 0 or non-finite (the recurrence cannot continue)."""
    f = np.asarray(f, dtype=np.float64)
    c = np.zeros_like(f)
    r = f.copy()
    p = r.copy()
    rr = float(r @ r)
    fn = math.sqrt(float(f @ f))
    status = "not_converged"
    k = 0
    if fn == 0.0:
        return CGResult(c, 0, 0.0, "ok")
    while k < maxit:
        if math.sqrt(rr) <= rtol * fn:
            status = "ok"
            break
        Ap = apply(p) + lam * p
        pAp = float(p @ Ap)
        if pAp == 0.0 or not math.isfinite(pAp):
            status = "breakdown"
            break
        a = rr / pAp
        c = c + a * p
        r = r - a * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
    else:
        if math.sqrt(rr) <= rtol * fn:
            status = "ok"
    true_r = f - (apply(c) + lam * c)
    return CGResult(c, k, math.sqrt(float(true_r @ true_r)) / fn, status)


def rel_err(y: np.ndarray, yref: np.ndarray) -> float:
    """max over RHS columns of ||y - y_ref||_2 / ||y_ref||_2."""
    y = np.atleast_2d(y)
    yref = np.atleast_2d(yref)
    num = np.sqrt(np.sum((y - yref) ** 2, axis=1))
    den = np.sqrt(np.sum(yref ** 2, axis=1))
    den[den == 0] = 1.0
    return float(np.max(num / den))
