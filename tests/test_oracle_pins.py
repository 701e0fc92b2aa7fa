"""Pins of the FP64 oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms
printed in the paper, library routines (numpy Legendre/Gauss quadrature,
scipy's pivoted QR and barycentric interpolation, scikit-learn's Matern/RBF
kernels), invariants of the method, and brute force on tiny inputs.
"""
import itertools
import math
import os

import numpy as np
import pytest

import dwfmm_inputs as di
from oracle import dwfmm_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Index sets (Sec. 4, Sec. 6.1)
# --------------------------------------------------------------------------

def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "sec6_1_counts.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, d, q, cnt = line.split()
            rows.append((kind, int(d), int(q), int(cnt)))
    return rows


@pytest.mark.parametrize("row", _golden_counts())
def test_sec61_closed_form_counts(row):
    kind, d, q, cnt = row
    if kind == "TPI":
        assert o.tensor_index_count(q, d) == cnt == (q + 1) ** d
    else:
        assert math.comb(q + d, d) == cnt
        if cnt <= 100000:
            assert len(o.index_set(np.ones(d), q)) == cnt


@pytest.mark.parametrize("d,q", [(1, 5), (2, 7), (3, 4), (5, 3), (6, 2)])
def test_total_degree_equals_binomial(d, q):
    assert len(o.index_set(np.ones(d), q)) == math.comb(q + d, d)


def test_index_set_brute_force_noninteger_weights():
    rng = np.random.default_rng(11)
    for _ in range(5):
        d = int(rng.integers(1, 5))
        w = rng.uniform(0.3, 3.0, size=d)
        q = float(rng.uniform(1.0, 5.0))
        got = {tuple(a) for a in o.index_set(w, q)}
        bound = [int(q / wk) + 1 for wk in w]
        ref = {a for a in itertools.product(*[range(b + 1) for b in bound])
               if float(np.dot(w, a)) <= q + 1e-9}
        assert got == ref


def test_index_set_small_workload_hand_count():
    # alpha_1 + 2 alpha_2 + 4 alpha_3 + 8 alpha_4 <= 4: alpha_4 = 0;
    # alpha_3 = 1 -> 1 index; alpha_3 = 0 -> 5 + 3 + 1 = 9; total 10.
    lam = o.index_set(o.weights_inv_gamma([1, .5, .25, .125]), 4)
    assert lam.shape == (10, 4)
    assert [0, 0, 1, 0] in lam.tolist()
    assert [4, 0, 0, 0] in lam.tolist()


def test_index_set_is_downward_closed_and_lexicographic():
    w = o.weights_inv_gamma(di.gamma_sqrt_half(10))
    lam = o.index_set(w, 8.0)
    s = {tuple(a) for a in lam}
    for a in lam:
        for k in range(len(a)):
            if a[k] > 0:
                b = list(a)
                b[k] -= 1
                assert tuple(b) in s
    assert [tuple(a) for a in lam] == sorted(tuple(a) for a in lam)


def test_sec61_wtdi_structure():
    """Sec. 6.1: WTDI needs far fewer points than TDI, grows with d and q,
    and shrinks as tau_k = k^r grows faster (r = 2, 3, 4)."""
    def cnt(d, q, r):
        tau = np.array([float(k) ** r for k in range(1, d + 1)])
        return len(o.index_set(o.weights_log_rho(tau), q))
    for r in (2, 3, 4):
        prev = 0
        for d in (2, 5, 10, 20):
            c = cnt(d, 6, r)
            assert c >= prev
            prev = c
        assert cnt(20, 10, r) >= cnt(20, 6, r)
    for d in (5, 10, 20):
        assert cnt(d, 8, 2) >= cnt(d, 8, 3) >= cnt(d, 8, 4)
        assert cnt(d, 8, 2) < math.comb(8 + d, d)


# --------------------------------------------------------------------------
# Weights (Lemma 4.1, Theorem 4.6, Sec. 6.2)
# --------------------------------------------------------------------------

def test_rho_identity_and_normalisation():
    tau = np.array([0.0, 0.1, 1.0, 7.5, 100.0])
    rho = o.rho_of_tau(tau)
    # rho = 2 tau + sqrt(1 + 4 tau^2)  <=>  rho - 1/rho = 4 tau, rho >= 1
    np.testing.assert_allclose(rho - 1.0 / rho, 4 * tau, rtol=0, atol=1e-12)
    assert rho[0] == 1.0
    w = o.weights_paper_normalised(np.array([1.0, 0.25, 1 / 9.0]), 0.5)
    assert abs(w[0] - 1.0) < 1e-15          # omega_1 = 1 (Sec. 6.2)
    assert np.all(np.diff(w) > 0)            # shorter edges -> larger weights
    np.testing.assert_allclose(o.weights_inv_gamma([0.5, 0.25, 0.125]), [1, 2, 4])


def _golden_weights():
    rows = []
    with open(os.path.join(GOLDEN, "sec6_2_weights.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, rest = line.split(None, 1)
            rows.append((kind, rest))
    return rows


def test_weights_match_hand_worked_values():
    """Sec. 6.2 rule and the unnormalised omega_k = log rho_k of Theorem 4.6
    against values worked by hand from the surds rho(tau) (golden file)."""
    rows = _golden_weights()
    assert sum(k == "paper" for k, _ in rows) == 2 and sum(k == "logrho" for k, _ in rows) == 2
    for kind, rest in rows:
        if kind == "paper":
            lhs, rhs = rest.split(";")
            eta, *b = [float(v) for v in lhs.split()]
            want = np.array([float(v) for v in rhs.split()])
            np.testing.assert_allclose(o.weights_paper_normalised(np.array(b), eta), want, rtol=0, atol=2e-15)
        else:
            tau, want = [float(v) for v in rest.split()]
            np.testing.assert_allclose(o.weights_log_rho(np.array([tau])), [want], rtol=0, atol=2e-15)


def test_planted_inverted_tau_is_caught(monkeypatch):
    """tau_k = eta / b_k instead of 1 / (eta b_k) keeps omega_1 = 1 and the
    monotone order, but not the hand-worked values."""
    def bad(b, eta):
        b = np.asarray(b, dtype=np.float64)
        tau = eta / b
        return np.log(math.e * o.rho_of_tau(tau) / o.rho_of_tau(tau[0]))
    monkeypatch.setattr(o, "weights_paper_normalised", bad)
    with pytest.raises(AssertionError):
        test_weights_match_hand_worked_values()


# --------------------------------------------------------------------------
# Legendre basis (Sec. 5.2)
# --------------------------------------------------------------------------

def test_legendre_orthonormal_gauss_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(30)
    t = 0.5 * (xg + 1.0)
    wt = 0.5 * wg
    P = o.legendre_hat(12, t)
    G = (P * wt[None, :]) @ P.T
    np.testing.assert_allclose(G, np.eye(13), atol=1e-13)


def test_legendre_matches_numpy_legval():
    t = np.linspace(0, 1, 37)
    P = o.legendre_hat(9, t)
    for j in range(10):
        c = np.zeros(j + 1)
        c[j] = 1.0
        ref = math.sqrt(2 * j + 1) * np.polynomial.legendre.legval(2 * t - 1, c)
        np.testing.assert_allclose(P[j], ref, atol=1e-13)


def test_tensor_basis_orthonormal_on_cube():
    lam = o.index_set([1.0, 1.5, 2.0], 4.0)
    xg, wg = np.polynomial.legendre.leggauss(8)
    t = 0.5 * (xg + 1)
    wt = 0.5 * wg
    T = np.array(list(itertools.product(t, t, t)))
    W = np.array([a * b * c for a, b, c in itertools.product(wt, wt, wt)])
    B = o.basis_eval(lam, T)
    np.testing.assert_allclose((B * W[:, None]).T @ B, np.eye(len(lam)), atol=1e-12)


# --------------------------------------------------------------------------
# Halton and approximate Fekete points (Sec. 5.4)
# --------------------------------------------------------------------------

def test_halton_van_der_corput_values():
    assert o.first_primes(10) == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    H = o.halton(8, 2)
    np.testing.assert_array_equal(H[:, 0], [1/2, 1/4, 3/4, 1/8, 5/8, 3/8, 7/8, 1/16])
    np.testing.assert_array_equal(H[:5, 1], [1/3, 2/3, 1/9, 4/9, 7/9])


def test_cpqr_matches_lapack_pivoting():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    for w, q, d in [([1.0, 2.0, 4.0, 8.0], 4.0, 4),
                    (o.weights_inv_gamma(di.gamma_inverse_square(8)), 6.0, 8),
                    (o.weights_inv_gamma(di.gamma_sqrt_half(10)), 8.0, 10)]:
        lam = o.index_set(w, q)
        n = len(lam)
        H = o.halton(o.halton_count(n), d)
        A = o.basis_eval(lam, H).T
        ours = o.greedy_cpqr(A)
        _, _, piv = scipy_linalg.qr(A, pivoting=True, mode="economic")
        assert ours == [int(p) for p in piv[:n]]


def test_unisolvent_nodes_reproduce_polynomials():
    rng = np.random.default_rng(5)
    for w, q in [([1, 2, 4, 8], 4.0), (list(o.weights_inv_gamma(di.gamma_sqrt_half(10))), 8.0)]:
        ex = o.make_expansion(np.array(w, dtype=float), q)
        n, d = ex.Lam.shape
        assert np.linalg.matrix_rank(ex.V) == n
        coef = rng.standard_normal(n)
        vals = ex.V @ coef                          # polynomial at the nodes
        rec = np.linalg.solve(ex.V, vals)
        T = rng.random((50, d))
        p_true = o.basis_eval(ex.Lam, T) @ coef
        p_int = o.basis_eval(ex.Lam, T) @ rec
        assert np.max(np.abs(p_true - p_int)) <= 1e-12 * max(1.0, np.max(np.abs(p_true)))


def test_one_dimensional_case_is_lagrange_interpolation():
    interp = pytest.importorskip("scipy.interpolate")
    q = 7
    ex = o.make_expansion(np.array([1.0]), q)
    xi = ex.nodes[:, 0]
    assert len(np.unique(xi)) == q + 1
    f = lambda t: np.cos(3 * t) + t ** 2
    t = np.linspace(0, 1, 41)
    ours = o.basis_eval(ex.Lam, t[:, None]) @ np.linalg.solve(ex.V, f(xi))
    ref = interp.BarycentricInterpolator(xi, f(xi))(t)
    np.testing.assert_allclose(ours, ref, atol=1e-12)


def test_lebesgue_constant_estimate_reported():
    ex = o.make_expansion(np.array([1.0, 2.0, 4.0, 8.0]), 4.0)
    T = o.halton(4000, 4, start=5000)
    Lag = np.linalg.solve(ex.V.T, o.basis_eval(ex.Lam, T).T).T   # Lagrange values
    leb = np.max(np.sum(np.abs(Lag), axis=1))
    # Fekete points give L <= |Lambda| (Sec. 5.4); approximate ones stay close.
    assert 1.0 <= leb <= 4 * ex.n


# --------------------------------------------------------------------------
# Kernels: library forms
# --------------------------------------------------------------------------

def test_kernels_match_scikit_learn():
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(3)
    X = rng.random((20, 3))
    Y = rng.random((15, 3))
    for sigma in (1.0, 0.37):
        np.testing.assert_allclose(o.kernel_matrix("matern32", X, Y, sigma),
                                   kern.Matern(length_scale=sigma, nu=1.5)(X, Y), rtol=1e-13)
        np.testing.assert_allclose(o.kernel_matrix("exp", X, Y, sigma),
                                   kern.Matern(length_scale=sigma, nu=0.5)(X, Y), rtol=1e-13)
        np.testing.assert_allclose(o.kernel_matrix("gauss", X, Y, sigma),
                                   kern.RBF(length_scale=sigma)(X, Y), rtol=1e-13)


# --------------------------------------------------------------------------
# Tree and lists (Sec. 5.1, Eq. (5.1))
# --------------------------------------------------------------------------

def _small(n=2000, d=4, seed=0):
    w = di.scaled(di.small_exp_d4(), n)
    w.seed = seed
    return di.sites(w)


def test_tree_invariants():
    X = _small(2000)
    tr = o.build_tree(X, 64)
    assert tr.depth == o.tree_depth(2000, 64) == 5
    assert sorted(tr.perm.tolist()) == list(range(2000))
    for j in range(tr.depth + 1):
        f, l = tr.level_range(j)
        sizes = tr.end[f:l] - tr.begin[f:l]
        assert sizes.max() - sizes.min() <= 1 and sizes.sum() == 2000
    f, l = tr.level_range(tr.depth)
    assert np.all(tr.end[f:l] - tr.begin[f:l] <= 64)
    for c in range((1 << tr.depth) - 1):
        c1, c2 = 2 * c + 1, 2 * c + 2
        assert tr.begin[c1] == tr.begin[c] and tr.end[c2] == tr.end[c]
        assert tr.end[c1] == tr.begin[c2]
        assert tr.end[c1] - tr.begin[c1] == -(-(tr.end[c] - tr.begin[c]) // 2)
        k = int(np.argmax(tr.hi[c] - tr.lo[c]))
        a = X[tr.perm[tr.begin[c1]:tr.end[c1]], k]
        b = X[tr.perm[tr.begin[c2]:tr.end[c2]], k]
        assert a.max() <= b.min()                   # split along the longest edge
        P = X[tr.perm[tr.begin[c]:tr.end[c]]]
        np.testing.assert_array_equal(tr.lo[c], P.min(0))
        np.testing.assert_array_equal(tr.hi[c], P.max(0))


def test_lists_partition_matrix_exactly_once():
    X = _small(700)
    tr = o.build_tree(X, 24)
    ls = o.build_lists(tr, 1.0)
    cover = np.zeros((700, 700), dtype=np.int64)
    blocks = [tuple(p) for lvl in ls.far for p in lvl] + [tuple(p) for p in ls.near]
    for (t, s) in blocks:
        cover[tr.begin[t]:tr.end[t], tr.begin[s]:tr.end[s]] += 1
    assert np.all(cover == 1)
    fs = {tuple(p) for lvl in ls.far for p in lvl}
    assert fs == {(s, t) for (t, s) in fs}
    assert {tuple(p) for p in ls.near} == {(s, t) for (t, s) in ls.near}
    # every leaf is near itself (a cluster is never admissible with itself):
    # with the symmetry above, the upper entries (t, s >= t) number
    # (|near| + leaves) / 2, which the symmetric float64 near field relies on
    leaves = set(range(*tr.level_range(tr.depth)))
    assert all((t, t) in {tuple(p) for p in ls.near} for t in leaves)
    assert sum(1 for (t, s) in ls.near if s >= t) * 2 == len(ls.near) + len(leaves)


def test_far_pairs_admissible_parents_not_by_euclid():
    X = _small(900)
    tr = o.build_tree(X, 32)
    eta = 1.0
    ls = o.build_lists(tr, eta)

    def adm_sqrt(a, b):
        gap = np.maximum(0, np.maximum(tr.lo[b] - tr.hi[a], tr.lo[a] - tr.hi[b]))
        dist = np.linalg.norm(gap)
        da = np.linalg.norm(tr.hi[a] - tr.lo[a])
        db = np.linalg.norm(tr.hi[b] - tr.lo[b])
        return dist > 0 and dist >= eta * max(da, db)

    for j, lvl in enumerate(ls.far):
        for (t, s) in lvl:
            assert adm_sqrt(t, s)
            if j > 0:
                assert not adm_sqrt((t - 1) // 2, (s - 1) // 2)
    for (t, s) in ls.near:
        assert not adm_sqrt(t, s)


# --------------------------------------------------------------------------
# Nested bases and the matvec (Sec. 5.2, Eq. (5.4), Sec. 5.3)
# --------------------------------------------------------------------------

def test_two_scale_relation_exact():
    X = _small(600)
    pb = o.make_problem(X, "exp", [1.0, 2.0, 4.0, 8.0], 4.0, 40, 1.0)
    tr = pb.tree
    for c in range(7):
        Pn = o.cluster_basis(pb.exp_, tr, c, X)
        stacked = np.vstack([o.cluster_basis(pb.exp_, tr, ch, X) @ o.transfer_matrix(pb.exp_, tr, ch)
                             for ch in (2 * c + 1, 2 * c + 2)])
        np.testing.assert_allclose(stacked, Pn, atol=1e-12 * max(1.0, np.abs(Pn).max()))


def test_single_leaf_is_exact():
    X = _small(50)
    f = np.random.default_rng(1).standard_normal((2, 50))
    pb = o.make_problem(X, "matern32", [1.0, 2.0, 4.0, 8.0], 4.0, 64, 1.0)
    assert pb.tree.depth == 0 and len(pb.lists.near) == 1
    y = o.fmm_matvec(pb, f)
    assert o.rel_err(y, o.dense_matvec("matern32", X, f)) <= 1e-14


def test_nested_equals_explicit_and_symmetric():
    X = _small(400)
    f = np.random.default_rng(2).standard_normal((3, 400))
    pb = o.make_problem(X, "gauss", [1.0, 1.5, 2.0, 3.0], 5.0, 20, 1.0)
    Kt = o.assemble_ktilde(pb)
    assert np.max(np.abs(Kt - Kt.T)) <= 1e-13
    y = o.fmm_matvec(pb, f)
    assert o.rel_err(y, (Kt @ f.T).T) <= 1e-12
    a, b = f[0], f[1]
    ya = o.fmm_matvec(pb, a[None])[0]
    yb = o.fmm_matvec(pb, b[None])[0]
    assert abs(b @ ya - a @ yb) <= 1e-13 * np.linalg.norm(a) * np.linalg.norm(ya)


def test_error_decays_exponentially_in_q():
    """Thm 4.6 / Cor. 4.9 / Cor. 5.7: compression error decays exponentially in q."""
    X = _small(1024)
    f = np.random.default_rng(3).standard_normal((1, 1024))
    ref = o.dense_matvec("gauss", X, f)
    errs = []
    for q in (1, 2, 3, 4, 5, 6):
        pb = o.make_problem(X, "gauss", np.ones(4), q, 32, 1.0)
        errs.append(o.rel_err(o.fmm_matvec(pb, f), ref))
    slope = np.polyfit(np.arange(1, 7), np.log(errs), 1)[0]
    assert slope < -1.0
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 1e-4


def test_error_roughly_independent_of_n():
    """Cor. 5.7 (quasi-uniform sites): the relative error does not grow with N."""
    errs = []
    for n in (1024, 4096):
        X = _small(n, seed=7)
        f = np.random.default_rng(4).standard_normal((1, n))
        pb = o.make_problem(X, "matern32", [1.0, 2.0, 4.0, 8.0], 4.0, 32, 1.0)
        errs.append(o.rel_err(o.fmm_matvec(pb, f), o.dense_matvec("matern32", X, f)))
    assert errs[1] < 3.0 * errs[0]


def test_leaf_restricted_matvec_equals_full():
    X = _small(800)
    f = np.random.default_rng(5).standard_normal((2, 800))
    pb = o.make_problem(X, "exp", [1.0, 2.0, 4.0, 8.0], 4.0, 25, 1.0)
    y = o.fmm_matvec(pb, f)
    tr = pb.tree
    f0, l0 = tr.level_range(tr.depth)
    leaves = [f0, f0 + 5, l0 - 1]
    part = o.fmm_matvec_leaves(pb, f, leaves)
    for c in leaves:
        idx = tr.perm[tr.begin[c]:tr.end[c]]
        np.testing.assert_allclose(part[c], y[:, idx].T, rtol=1e-13, atol=1e-13)


def test_cg_matches_dense_solve():
    X = _small(300)
    pb = o.make_problem(X, "matern32", [1.0, 2.0, 4.0, 8.0], 4.0, 20, 1.0)
    Kt = o.assemble_ktilde(pb)
    f = np.random.default_rng(6).standard_normal(300)
    # compression can make K_tilde slightly indefinite; shift past its spectrum
    lam = 1e-2 + 2.0 * max(0.0, -float(np.linalg.eigvalsh(Kt)[0]))
    res = o.cg(lambda v: Kt @ v, f, lam, 1e-10, 2000)
    assert res.status == "ok" and res.relres <= 1e-9
    ref = np.linalg.solve(Kt + lam * np.eye(300), f)
    kappa = np.linalg.cond(Kt + lam * np.eye(300))
    assert np.linalg.norm(res.c - ref) / np.linalg.norm(ref) <= kappa * 1e-10


def test_cg_breakdown_and_maxit():
    # zero curvature: p = f = e1 and e1^T A e1 = 0 -- the recurrence cannot continue
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    res = o.cg(lambda v: A @ v, np.array([1.0, 0.0]), 0.0, 1e-12, 10)
    assert res.status == "breakdown"
    # negative curvature is tolerated: diag(1, -1, 2) c = e2 is solved in one step (c = -e2)
    A = np.diag([1.0, -1.0, 2.0])
    res = o.cg(lambda v: A @ v, np.array([0.0, 1.0, 0.0]), 0.0, 1e-12, 10)
    assert res.status == "ok" and res.iters == 1
    np.testing.assert_allclose(res.c, [0.0, -1.0, 0.0])
    B = np.diag(np.linspace(1, 1e4, 50))
    res = o.cg(lambda v: B @ v, np.ones(50), 0.0, 1e-14, 3)
    assert res.status == "not_converged" and res.iters == 3


# --------------------------------------------------------------------------
# Planted mistakes: each plausible slip in the oracle trips a pin above.
# --------------------------------------------------------------------------

def test_planted_transposed_transfer_is_caught(monkeypatch):
    X = _small(400)
    f = np.random.default_rng(2).standard_normal((1, 400))
    pb = o.make_problem(X, "gauss", [1.0, 1.5, 2.0, 3.0], 5.0, 20, 1.0)
    Kt = o.assemble_ktilde(pb)
    good = o.problem_transfer
    pb.cache.clear()
    monkeypatch.setattr(o, "problem_transfer", lambda p_, c: good(p_, c).T)
    assert o.rel_err(o.fmm_matvec(pb, f), (Kt @ f.T).T) > 1e-6


def test_planted_legendre_sign_is_caught(monkeypatch):
    good = o.legendre_hat

    def bad(jmax, t):
        P = good(jmax, t)
        if jmax >= 2:
            P[2] = -P[2]
        return P
    monkeypatch.setattr(o, "legendre_hat", bad)
    with pytest.raises(AssertionError):
        test_legendre_matches_numpy_legval()


def test_planted_dropped_far_level_is_caught():
    X = _small(700)
    tr = o.build_tree(X, 24)
    ls = o.build_lists(tr, 1.0)
    j = int(np.argmax([len(lvl) for lvl in ls.far]))
    assert len(ls.far[j]) > 0
    ls.far[j] = ls.far[j][:0]
    cover = np.zeros((700, 700), dtype=np.int64)
    for lvl in ls.far:
        for (t, s) in lvl:
            cover[tr.begin[t]:tr.end[t], tr.begin[s]:tr.end[s]] += 1
    for (t, s) in ls.near:
        cover[tr.begin[t]:tr.end[t], tr.begin[s]:tr.end[s]] += 1
    assert not np.all(cover == 1)


def test_vectorised_admissibility_equals_scalar_rule():
    X = _small(1500, seed=3)
    tr = o.build_tree(X, 20)
    rng = np.random.default_rng(0)
    t = rng.integers(0, tr.nclusters, 4000)
    s = rng.integers(0, tr.nclusters, 4000)
    for eta in (0.5, 1.0, 2.0):
        vec = o.admissible_pairs(tr.lo, tr.hi, t, s, eta)
        ref = [o.admissible(tr.lo[a], tr.hi[a], tr.lo[b], tr.hi[b], eta) for a, b in zip(t, s)]
        assert vec.tolist() == ref


# ---------------------------------------------------------------------------
# Tensor-product index set (Sec. 6.1's TPI, max_k omega_k alpha_k <= q)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,q", [(1, 5), (2, 3), (3, 2), (4, 1), (5, 0)])
def test_tensor_set_count_is_q_plus_one_to_the_d(d, q):
    """Sec. 6.1: |{alpha : ||alpha||_inf <= q}| = (q+1)^d."""
    lam = o.index_set(np.ones(d), q, "tensor")
    assert lam.shape == (o.tensor_index_count(q, d), d) == ((q + 1) ** d, d)
    assert len({tuple(a) for a in lam}) == len(lam)
    assert lam.max(initial=0) <= q


def test_tensor_set_anisotropic_count_and_order():
    w, q = [1.0, 2.0, 0.7], 3.0
    lam = o.index_set(w, q, "tensor")
    # per coordinate the a >= 0 with omega_k a <= q: 0..3, 0..1, 0..4
    assert len(lam) == 4 * 2 * 5
    assert [tuple(a) for a in lam] == sorted(tuple(a) for a in lam)     # lexicographic
    brute = [a for a in itertools.product(range(6), repeat=3) if max(wk * ak for wk, ak in zip(w, a)) <= q]
    assert sorted(tuple(a) for a in lam) == sorted(brute)


def test_total_degree_set_is_inside_tensor_set_and_equal_in_one_dimension():
    for w, q in [([1.0, 1.0, 1.0], 3.0), ([1.0, 2.0, 4.0, 8.0], 4.0), ([0.5, 1.5], 2.0)]:
        td = {tuple(a) for a in o.index_set(w, q)}
        tp = {tuple(a) for a in o.index_set(w, q, "tensor")}
        assert td <= tp and (len(w) == 1 or td != tp)
    np.testing.assert_array_equal(o.index_set([1.0], 6.0), o.index_set([1.0], 6.0, "tensor"))


def test_tensor_expansion_reproduces_a_mixed_degree_monomial():
    """x1^q x2^q lies in the tensor-product space but not in the total-degree
    space of degree q: the tensor expansion interpolates it exactly, the
    total-degree one does not."""
    q = 3
    f = lambda X: X[:, 0] ** q * X[:, 1] ** q
    rng = np.random.default_rng(11)
    T = rng.random((40, 2))
    errs = {}
    for shape in ("tensor", "total"):
        ex = o.make_expansion(np.ones(2), float(q), shape=shape)
        coef = np.linalg.solve(ex.V, f(ex.nodes))
        errs[shape] = np.max(np.abs(o.basis_eval(ex.Lam, T) @ coef - f(T)))
    assert errs["tensor"] <= 1e-12
    assert errs["total"] > 1e-4
