"""Pins for the FP64 oracle: closed forms, library routines and invariants.

Each test ties the oracle to something other than itself, so that a dropped
term, a wrong sign or a transposed message index fails at least one of them:

* the 2-node graph worked by hand (tests/golden/n2_closed_form.json),
* trees, where GaBP is exact in means and precisions after diameter rounds,
* dense diagonally dominant matrices, where the converged means solve Q mu = b
  (numpy's LAPACK solve),
* equality of the information form, the printed form of Algorithm 2 and
  Algorithm 1 round by round,
* invariants (precisions independent of b, linearity in b, permutation
  equivariance, message fixed-point equations),
* the RBF matrix against scipy's pairwise distances and hand values,
* the decision function against the SVM matrix, the dual objective at the
  optimum, matrix-free CG against a dense solve, the box-QP brute force
  against scipy's bounded minimiser and its KKT conditions.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dd_matrix(n, seed, delta=0.2, density=1.0):
    """Random symmetric matrix with a dominant diagonal, mixed signs."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (n, n))
    if density < 1.0:
        A *= rng.uniform(0, 1, (n, n)) < density
    A = np.triu(A, 1)
    A = A + A.T
    d = (1 + delta) * np.abs(A).sum(1) + rng.uniform(0.1, 1.0, n)
    A[np.diag_indices(n)] = d
    return A


# ---------------------------------------------------------------- 2-node graph
def test_two_node_closed_form():
    g = json.load(open(os.path.join(GOLD, "n2_closed_form.json")))
    Q, b = np.array(g["Q"]), np.array(g["b"])
    r0 = oracle.gabp(Q, b, iters=0)
    np.testing.assert_allclose(r0.Pt, g["t0"]["Ptilde"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r0.mu, g["t0"]["mutilde"], rtol=0, atol=1e-15)
    for t in range(1, 6):
        r = oracle.gabp(Q, b, iters=t, keep_messages=True)
        np.testing.assert_allclose(r.Pt, g["t_ge_1"]["Ptilde"], rtol=1e-15)
        np.testing.assert_allclose(r.mu, g["t_ge_1"]["mutilde"], rtol=1e-15)
        assert r.rinf <= 1e-15
        m = g["messages_t_ge_1"]
        # Pin[i, k] = P_ki: message node1 -> node2 sits in row 1 (0-based).
        assert r.Pin[1, 0] == pytest.approx(m["P_12"], rel=1e-15)
        assert r.Pin[0, 1] == pytest.approx(m["P_21"], rel=1e-15)
        assert r.Hin[1, 0] == pytest.approx(m["H_12"], rel=1e-15)
        assert r.Hin[0, 1] == pytest.approx(m["H_21"], rel=1e-15)
    # with a tolerance, the first converged round is t = 1
    r = oracle.gabp(Q, b, iters=50, tol=1e-12)
    assert r.kstar == 1


# ----------------------------------------------------------------------- trees
def _chain(n, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    off = rng.uniform(-1, 1, n - 1)
    A[np.arange(n - 1), np.arange(1, n)] = off
    A[np.arange(1, n), np.arange(n - 1)] = off
    A[np.diag_indices(n)] = np.abs(A).sum(1) * rng.uniform(0.8, 1.5, n) + 0.2
    return A


def _star(n, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    off = rng.uniform(-1, 1, n - 1)
    A[0, 1:] = off
    A[1:, 0] = off
    A[np.diag_indices(n)] = np.abs(A).sum(1) * 1.3 + 0.1
    return A


@pytest.mark.parametrize("make,n,diam", [(_chain, 9, 8), (_star, 12, 2)])
def test_tree_exact_means_and_precisions(make, n, diam):
    Q = make(n, 3)
    assert np.all(np.linalg.eigvalsh(Q) > 0)
    b = np.random.default_rng(4).standard_normal(n)
    inv = np.linalg.inv(Q)
    r = oracle.gabp(Q, b, iters=diam)
    np.testing.assert_allclose(r.mu, inv @ b, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r.Pt, 1.0 / np.diag(inv), rtol=1e-12)
    # before `diam` rounds the far ends have not heard from each other yet
    r_early = oracle.gabp(Q, b, iters=diam - 1)
    assert np.max(np.abs(r_early.mu - inv @ b)) > 1e-9


# ------------------------------------------------------- dense DD fixed point
@pytest.mark.parametrize("n,seed", [(5, 1), (17, 2), (64, 3)])
def test_dense_fixed_point_is_linear_solve(n, seed):
    Q = _dd_matrix(n, seed)
    b = np.ones(n)
    ref = np.linalg.solve(Q, b)
    r = oracle.gabp(Q, b, iters=2000, tol=1e-13)
    assert r.kstar < 2000
    np.testing.assert_allclose(r.mu, ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(oracle.cholesky_solve(Q, b), ref, rtol=1e-12, atol=1e-14)
    # residual history is what it claims: ||b - Q mu||_inf at kstar
    assert r.rinf == pytest.approx(np.max(np.abs(b - Q @ r.mu)), rel=1e-6, abs=1e-13)


def test_loopy_precisions_are_not_exact():
    """On a loopy graph only the means are exact (Section 2 convergence)."""
    Q = _dd_matrix(10, 5)
    r = oracle.gabp(Q, np.ones(10), iters=3000, tol=1e-14)
    inv = np.linalg.inv(Q)
    np.testing.assert_allclose(r.mu, inv @ np.ones(10), rtol=1e-10)
    assert np.max(np.abs(r.Pt - 1.0 / np.diag(inv)) / r.Pt) > 1e-6


# ------------------------------------------------------------ form equivalence
@pytest.mark.parametrize("n,seed,density", [(6, 7, 1.0), (12, 8, 1.0), (15, 9, 0.5)])
@pytest.mark.parametrize("iters", [1, 2, 3, 7])
def test_three_forms_agree_round_by_round(n, seed, density, iters):
    Q = _dd_matrix(n, seed, density=density)
    b = np.random.default_rng(seed).standard_normal(n)
    r = oracle.gabp(Q, b, iters=iters)
    mu_l, Pt_l = oracle.gabp_literal(Q, b, iters=iters)
    mu_1, Pt_1 = oracle.gabp_alg1(Q, b, iters=iters)
    np.testing.assert_allclose(r.mu, mu_l, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r.Pt, Pt_l, rtol=1e-12)
    np.testing.assert_allclose(r.mu, mu_1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r.Pt, Pt_1, rtol=1e-12)


# ------------------------------------------------------------------ invariants
def test_precisions_do_not_depend_on_b_and_means_are_linear_in_b():
    Q = _dd_matrix(20, 11)
    rng = np.random.default_rng(12)
    b1, b2 = rng.standard_normal(20), rng.standard_normal(20)
    for it in (1, 4, 9):
        r1 = oracle.gabp(Q, b1, iters=it)
        r2 = oracle.gabp(Q, b2, iters=it)
        r3 = oracle.gabp(Q, 2.0 * b1 - 3.0 * b2, iters=it)
        np.testing.assert_array_equal(r1.Pt, r2.Pt)
        np.testing.assert_allclose(r3.mu, 2.0 * r1.mu - 3.0 * r2.mu, rtol=1e-11, atol=1e-13)


def test_permutation_equivariance():
    Q = _dd_matrix(14, 13)
    b = np.random.default_rng(14).standard_normal(14)
    perm = np.random.default_rng(15).permutation(14)
    r = oracle.gabp(Q, b, iters=6)
    rp = oracle.gabp(Q[np.ix_(perm, perm)], b[perm], iters=6)
    np.testing.assert_allclose(rp.mu, r.mu[perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rp.Pt, r.Pt[perm], rtol=1e-12)


def test_message_fixed_point_equations_hold_at_convergence():
    n = 16
    Q = _dd_matrix(n, 21)
    b = np.ones(n)
    r = oracle.gabp(Q, b, iters=3000, tol=1e-14, keep_messages=True)
    Pin, Hin = r.Pin, r.Hin
    ht = b + (Hin.sum(1) - np.diag(Hin))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            cav = r.Pt[i] - Pin[i, j]            # P_{i\j} = Ptilde_i - P_ji
            assert cav > 0
            # message i->j is stored at Pin[j, i]
            assert Pin[j, i] == pytest.approx(-Q[i, j] ** 2 / cav, rel=1e-9)
            assert Hin[j, i] == pytest.approx(-Q[i, j] * (ht[i] - Hin[i, j]) / cav,
                                              rel=1e-8, abs=1e-14)


def test_pair_update_matches_one_round():
    n = 9
    Q = _dd_matrix(n, 31)
    b = np.ones(n)
    r1 = oracle.gabp(Q, b, iters=3, keep_messages=True)
    r2 = oracle.gabp(Q, b, iters=4, keep_messages=True)
    ht = b + (r1.Hin.sum(1) - np.diag(r1.Hin))
    for (i, j) in [(0, 1), (2, 7), (5, 8)]:
        msg = [r1.Pin[j, i], r1.Pin[i, j], r1.Hin[j, i], r1.Hin[i, j]]
        out = oracle.pair_update(Q[i, j], r1.Pt[i], ht[i], r1.Pt[j], ht[j], msg)
        np.testing.assert_allclose(out, [r2.Pin[j, i], r2.Pin[i, j], r2.Hin[j, i], r2.Hin[i, j]],
                                   rtol=1e-14)


def test_non_dominant_matrix_reports_numeric_failure():
    # Strongly coupled 3-cycle with a tiny diagonal: the cavity precision
    # P_ii + sum P_ki goes nonpositive in the first rounds.
    Q = np.array([[0.1, 1.0, 1.0], [1.0, 0.1, 1.0], [1.0, 1.0, 0.1]])
    with pytest.raises(oracle.OracleError):
        oracle.gabp(Q, np.ones(3), iters=20)


# ------------------------------------------------------------------ SVM matrix
def test_q_matches_scipy_rbf_and_hand_values():
    from scipy.spatial.distance import cdist

    p = workloads.two_gaussians(40, 5, seed=3)
    lam = 1.0 / p.n
    Q = oracle.build_q(p.X, p.y, p.gamma, p.C)
    K = np.exp(-p.gamma * cdist(p.X, p.X, "sqeuclidean"))
    Dm = np.outer(p.y, p.y) * (K + lam * lam)
    off = ~np.eye(p.n, dtype=bool)
    np.testing.assert_allclose(Q[off], Dm[off], rtol=1e-13)
    np.testing.assert_array_equal(Q, Q.T)
    # dominant rule: Q_ii = max(1 + lam^2 + 1/C, (1 + delta) sum_{j != i} |Q_ij|)
    R = np.abs(Q).sum(1) - np.diag(Q)
    floor = 1.0 + lam * lam + 1.0 / p.C
    np.testing.assert_allclose(np.diag(Q), np.maximum(1.1 * R, floor), rtol=1e-14)
    assert np.any(1.1 * R < floor) and np.any(1.1 * R > floor)   # both branches seen
    # soft2 rule: D_ii + 1/C
    Q2 = oracle.build_q(p.X, p.y, p.gamma, p.C, diag_rule=oracle.DIAG_SOFT2)
    np.testing.assert_allclose(np.diag(Q2), 1.0 + lam * lam + 1.0 / p.C, rtol=1e-15)
    # hand value: x=(0,0), x'=(1,0), gamma=1/2, y=(+1,-1), lambda=0.5
    q = oracle.q_offdiag([0.0, 0.0], [1.0, 0.0], 1.0, -1.0, 0.5, 0.5)
    assert q == pytest.approx(-(np.exp(-0.5) + 0.25), rel=1e-15)
    # translation invariance of the RBF kernel
    Qs = oracle.build_q(p.X + 3.25, p.y, p.gamma, p.C)
    np.testing.assert_allclose(Qs, Q, rtol=1e-12)
    # small-C floor of the diagonal rule
    assert oracle.q_diag(0.5, 0.1, 0.25) == pytest.approx(1.0 + 0.01 + 4.0)


def test_workload_solve_reaches_the_linear_solve():
    p = workloads.two_gaussians(300, 10, seed=5)
    Q, r = oracle.solve_svm(p.X, p.y, p.gamma, p.C, iters=400, tol=1e-10)
    assert r.kstar < 400
    ref = np.linalg.solve(Q, np.ones(p.n))
    np.testing.assert_allclose(r.mu, ref, rtol=1e-8, atol=1e-12)
    # residual decreases over the run (dominant diagonal: contraction)
    assert r.rhist[-1] < 1e-3 * r.rhist[0]


# ------------------------------------------------------------ decision / dual
def test_decision_matches_svm_matrix_on_training_points():
    p = workloads.two_gaussians(60, 4, seed=6)
    lam = 1.0 / p.n
    Q = oracle.build_q(p.X, p.y, p.gamma, p.C)
    alpha = np.random.default_rng(7).uniform(0, 1, p.n)
    f = oracle.decision(p.X, p.y, alpha, p.X, p.gamma)
    # f(x_k) = y_k (D alpha)_k with D = Q except D_kk = 1 + lambda^2
    D = Q.copy()
    D[np.diag_indices(p.n)] = 1.0 + lam * lam
    np.testing.assert_allclose(f, p.y * (D @ alpha), rtol=1e-12, atol=1e-13)
    from scipy.spatial.distance import cdist
    Xt = workloads.test_points(p, 7, seed=8)
    K = np.exp(-p.gamma * cdist(Xt, p.X, "sqeuclidean"))
    np.testing.assert_allclose(oracle.decision(p.X, p.y, alpha, Xt, p.gamma),
                               (K + lam * lam) @ (alpha * p.y), rtol=1e-12)


def test_dual_objective():
    Q = _dd_matrix(12, 41)
    h = np.random.default_rng(42).uniform(0, 1, 12)
    assert oracle.dual_objective(Q, h) == pytest.approx(h.sum() - 0.5 * h @ Q @ h, rel=1e-13)
    # at the unconstrained optimum a* = Q^-1 1 the value is 1/2 sum a*
    a = np.linalg.solve(Q, np.ones(12))
    assert oracle.dual_objective(Q, a) == pytest.approx(0.5 * a.sum(), rel=1e-12)


def test_matrix_free_cg_matches_dense_solve():
    p = workloads.mixture(150, 8, seed=9, C=2.0)
    Q = oracle.build_q(p.X, p.y, p.gamma, p.C)
    x, its = oracle.cg_rbf(p.X, p.y, p.gamma, p.C, rtol=1e-13)
    np.testing.assert_allclose(x, np.linalg.solve(Q, np.ones(p.n)), rtol=1e-9, atol=1e-13)
    row = oracle.q_row(p.X, p.y, 17, p.gamma, p.C)
    np.testing.assert_allclose(row, Q[17], rtol=1e-14)


def test_q_diag_all_rows():
    """The all-row diagonal pass: closed form on identical patterns (every
    K = 1, so R_i = (n - 1)(1 + lambda^2)), the dense matrix's diagonal and row
    sums otherwise, and the Varah bound it feeds (||Q^-1||_inf <= 1 /
    min_i (Q_ii - R_i) for strictly diagonally dominant Q)."""
    n, lam, C = 37, 1.0 / 37, 0.5
    X = np.tile(np.array([[0.3, -1.2, 2.0]]), (n, 1))
    y = np.where(np.arange(n) % 3 == 0, -1.0, 1.0)
    d, R = oracle.q_diag_all(X, y, 0.7, C)
    np.testing.assert_allclose(R, (n - 1) * (1 + lam * lam), rtol=1e-14)
    np.testing.assert_allclose(d, max(1 + lam * lam + 1 / C, 1.1 * (n - 1) * (1 + lam * lam)), rtol=1e-14)
    p = workloads.mixture(140, 9, seed=12, C=3.0)
    Q = oracle.build_q(p.X, p.y, p.gamma, p.C)
    d, R = oracle.q_diag_all(p.X, p.y, p.gamma, p.C)
    np.testing.assert_allclose(d, np.diag(Q), rtol=1e-13)
    np.testing.assert_allclose(R, np.abs(Q).sum(1) - np.abs(np.diag(Q)), rtol=1e-13)
    inv_norm = np.abs(np.linalg.inv(Q)).sum(1).max()
    assert inv_norm <= 1.0 / np.min(d - R) * (1 + 1e-12)


# ------------------------------------------------------------------ box QP
@pytest.mark.parametrize("n,seed,C", [(6, 51, 0.05), (9, 52, 0.3), (11, 53, 10.0)])
def test_boxqp_bruteforce_against_scipy_and_kkt(n, seed, C):
    from scipy.optimize import minimize

    p = workloads.two_gaussians(n, 3, seed=seed)
    Q = oracle.build_q(p.X, p.y, p.gamma, p.C, diag_rule=oracle.DIAG_SOFT2)
    a, nk = oracle.boxqp_bruteforce(Q, C)
    assert nk == 1          # strictly convex: exactly one KKT point
    g = Q @ a - 1.0
    assert np.all(a >= -1e-12) and np.all(a <= C + 1e-12)
    free = (a > 1e-9) & (a < C - 1e-9)
    assert np.all(np.abs(g[free]) < 1e-9)
    assert np.all(g[a <= 1e-9] >= -1e-9) and np.all(g[a >= C - 1e-9] <= 1e-9)
    res = minimize(lambda v: 0.5 * v @ Q @ v - v.sum(), np.full(n, C / 2),
                   jac=lambda v: Q @ v - 1.0, bounds=[(0, C)] * n, method="L-BFGS-B",
                   options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    np.testing.assert_allclose(a, res.x, atol=1e-6)


def test_boxqp_equals_clipped_gabp_when_inside_box():
    """When Q^-1 1 lies inside [0, C]^n, the box constraints are inactive and
    the paper's relaxation (Section 3) loses nothing: alpha_box = mu*."""
    p = workloads.two_gaussians(10, 4, seed=61)
    C = 10.0
    Q = oracle.build_q(p.X, p.y, p.gamma, C)
    r = oracle.gabp(Q, np.ones(p.n), iters=5000, tol=1e-14)
    if not np.all((r.mu > 0) & (r.mu < C)):
        pytest.skip("optimum not inside the box for this draw")
    a, _ = oracle.boxqp_bruteforce(Q, C)
    np.testing.assert_allclose(a, r.alpha(C), rtol=1e-9, atol=1e-12)


# ------------------------------------------------- kernel ridge regression task
def _rbf(A, B, gamma):
    from scipy.spatial.distance import cdist
    return np.exp(-gamma * cdist(A, B, "sqeuclidean"))


def test_krr_two_points_closed_form():
    """Section 1.2 with two points: (K + l I) c = t solved by hand."""
    X = np.array([[0.0, 0.0], [1.0, 2.0]])
    gamma, ridge = 0.3, 0.7
    k = np.exp(-gamma * 5.0)
    t = np.array([0.4, -1.3])
    det = (1 + ridge) ** 2 - k * k
    c = np.array([((1 + ridge) * t[0] - k * t[1]) / det, ((1 + ridge) * t[1] - k * t[0]) / det])
    Q, r = oracle.solve_krr(X, t, gamma, ridge, iters=5, tol=0.0, diag_rule=oracle.DIAG_SOFT2)
    np.testing.assert_allclose(Q, [[1 + ridge, k], [k, 1 + ridge]], rtol=1e-15)
    np.testing.assert_allclose(r.mu, c, rtol=1e-14)    # a tree: exact after one round


@pytest.mark.parametrize("n,m,seed", [(40, 3, 1), (120, 8, 2)])
def test_krr_fixed_point_is_ridge_solve(n, m, seed):
    """With a ridge large enough for diagonal dominance, GaBP converges to
    (K + ridge I)^-1 t, K from scipy's distances and the solve by LAPACK."""
    p = workloads.mixture(n, m, seed=seed)
    X = p.X.astype(np.float64)
    t = workloads.krr_targets(p, seed + 10).astype(np.float64)
    K = _rbf(X, X, p.gamma)
    ridge = 1.2 * (K.sum(1) - 1).max()
    ref = np.linalg.solve(K + ridge * np.eye(n), t)
    Q, r = oracle.solve_krr(X, t, p.gamma, ridge, iters=3000, tol=1e-13, diag_rule=oracle.DIAG_SOFT2)
    assert r.kstar < 3000
    np.testing.assert_allclose(Q, K + ridge * np.eye(n), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(r.mu, ref, rtol=1e-9, atol=1e-12)


def test_krr_dominant_rule_keeps_kernel_and_solves_its_matrix():
    """Dominant rule: the off-diagonal is the bare kernel (no labels, no bias),
    the diagonal at least 1 + ridge, and GaBP reaches that matrix's solve."""
    p = workloads.mixture(150, 6, seed=5)
    X = p.X.astype(np.float64)
    t = workloads.krr_targets(p, 6).astype(np.float64)
    Q, r = oracle.solve_krr(X, t, p.gamma, 0.5, iters=3000, tol=1e-12)
    off = ~np.eye(p.n, dtype=bool)
    np.testing.assert_allclose(Q[off], _rbf(X, X, p.gamma)[off], rtol=1e-13)
    assert np.all(np.diag(Q) >= 1.5 - 1e-12)
    np.testing.assert_allclose(r.mu, np.linalg.solve(Q, t), rtol=1e-9, atol=1e-12)


def test_krr_prediction_matches_section_1_2_formula():
    """f(x) = t^T (K + l I)^-1 k(x) (Section 1.2) equals sum_i c_i K(x_i, x)
    with the oracle's coefficients."""
    p = workloads.mixture(60, 4, seed=8)
    X = p.X.astype(np.float64)
    t = workloads.krr_targets(p, 9).astype(np.float64)
    K = _rbf(X, X, p.gamma)
    ridge = 1.2 * (K.sum(1) - 1).max()
    _, r = oracle.solve_krr(X, t, p.gamma, ridge, iters=3000, tol=1e-13, diag_rule=oracle.DIAG_SOFT2)
    Xt = workloads.test_points(p, 25, seed=10).astype(np.float64)
    f_ref = t @ np.linalg.solve(K + ridge * np.eye(p.n), _rbf(X, Xt, p.gamma))
    f = oracle.decision(X, np.ones(p.n), r.mu, Xt, p.gamma, lam=0.0)
    np.testing.assert_allclose(f, f_ref, rtol=1e-9, atol=1e-12)


# ------------------------------------------- block Gauss-Seidel (staged) schedule
def test_stage_bounds_balance_block_pairs():
    for nt, s in [(157, 4), (32, 2), (3, 4), (1, 2), (782, 8)]:
        B = oracle.stage_bounds(nt, s)
        assert B[0] == 0 and B[-1] == nt and all(B[k] <= B[k + 1] for k in range(s))
        tot = nt * (nt + 1) // 2
        for k in range(1, s):
            b = B[k]
            assert s * (b * (b + 1) // 2) >= k * tot                      # reaches its share ...
            assert b == 0 or s * ((b - 1) * b // 2) < k * tot             # ... and no earlier block does


@pytest.mark.parametrize("n,seed", [(17, 2), (64, 3), (130, 4)])
def test_staged_one_stage_is_the_synchronous_schedule(n, seed):
    Q = _dd_matrix(n, seed)
    b = np.random.default_rng(seed).standard_normal(n)
    for iters in (0, 1, 5):
        r1 = oracle.gabp(Q, b, iters=iters)
        r2 = oracle.gabp_staged(Q, b, iters=iters, stages=1, block=8)
        np.testing.assert_array_equal(r1.mu, r2.mu)
        np.testing.assert_array_equal(r1.Pt, r2.Pt)
    # a single block puts every pair in one stage, whatever the stage count
    r3 = oracle.gabp_staged(Q, b, iters=4, stages=4, block=n)
    np.testing.assert_array_equal(oracle.gabp(Q, b, iters=4).mu, r3.mu)


@pytest.mark.parametrize("n,seed,stages,block", [(64, 3, 2, 8), (130, 4, 4, 16), (200, 5, 8, 8)])
def test_staged_fixed_point_is_linear_solve(n, seed, stages, block):
    Q = _dd_matrix(n, seed)
    b = np.random.default_rng(seed + 1).standard_normal(n)
    r = oracle.gabp_staged(Q, b, iters=2000, tol=1e-13, stages=stages, block=block)
    assert r.kstar < 2000
    np.testing.assert_allclose(r.mu, np.linalg.solve(Q, b), rtol=1e-10, atol=1e-12)
    # the invariants of the synchronous schedule hold too
    r2 = oracle.gabp_staged(Q, 3.0 * b, iters=7, stages=stages, block=block)
    r1 = oracle.gabp_staged(Q, b, iters=7, stages=stages, block=block)
    np.testing.assert_allclose(r2.mu, 3.0 * r1.mu, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(r2.Pt, r1.Pt)


def test_staged_schedule_needs_fewer_rounds_on_the_svm_matrix():
    """Section 3.2's point that non-synchronous schedules converge faster, on
    a seeded SVM matrix of the mixture workload."""
    p = workloads.mixture(600, 16, seed=12, C=1.0)
    Q = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    k1 = oracle.gabp(Q, np.ones(p.n), iters=500, tol=1e-8).kstar
    k4 = oracle.gabp_staged(Q, np.ones(p.n), iters=500, tol=1e-8, stages=4, block=128).kstar
    assert k4 < k1 < 500


# ------------------------------------------------------------ tile-sparse kernel
def test_tile_sparse_matrix_pins():
    p = workloads.clustered_mixture(1500, 64, seed=3, gamma=0.15)
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    Qd = oracle.build_q(X, y, p.gamma, p.C)
    # a threshold below every entry keeps the dense matrix
    Q0, keep0 = oracle.build_q_tile_sparse(X, y, p.gamma, p.C, 0.0)
    np.testing.assert_array_equal(Q0, Qd)
    assert keep0.sum() == keep0.shape[0] * (keep0.shape[0] + 1) // 2
    tau = 1e-4
    Q, keep = oracle.build_q_tile_sparse(X, y, p.gamma, p.C, tau)
    assert 0 < (~keep[np.triu_indices(keep.shape[0], 1)]).sum()
    np.testing.assert_array_equal(Q, Q.T)
    off = ~np.eye(p.n, dtype=bool)
    kept = Q[off] != 0
    np.testing.assert_array_equal(Q[off][kept], Qd[off][kept])      # kept entries unchanged
    assert np.abs(Qd[off][~kept]).max() <= tau                       # dropped ones were small
    # the diagonal is the whole matrix's, so the sparse matrix stays diagonally dominant
    np.testing.assert_array_equal(np.diag(Q), np.diag(Qd))
    assert np.all(np.diag(Q) > np.abs(Q).sum(1) - np.diag(Q))
    # GaBP on the sparse matrix reaches its linear solve
    r = oracle.gabp(Q, np.ones(p.n), iters=500, tol=1e-12)
    assert r.kstar < 500
    np.testing.assert_allclose(r.mu, np.linalg.solve(Q, np.ones(p.n)), rtol=1e-9, atol=1e-12)


def test_oracle_builds_and_agrees_without_openmp(tmp_path):
    """The C oracle compiles without OpenMP (one thread) and its all-row
    diagonal pass gives the same values as the OpenMP build."""
    import ctypes
    import subprocess
    src = os.path.join(os.path.dirname(oracle.__file__), "gabp_oracle.c")
    so = str(tmp_path / "liboracle_serial.so")
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-Wno-unknown-pragmas",
                    "-fno-fast-math", "-ffp-contract=off", src, "-o", so, "-lm"], check=True)
    lib = ctypes.CDLL(so)
    assert lib.orc_threads() == 1
    rng = np.random.default_rng(4)
    X = rng.standard_normal((57, 5))
    y = np.where(rng.random(57) < 0.5, 1.0, -1.0)
    D = ctypes.POINTER(ctypes.c_double)
    d1, R1 = np.empty(57), np.empty(57)
    lib.orc_q_diag_all.argtypes = [D, D, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, D, D]
    rc = lib.orc_q_diag_all(X.ctypes.data_as(D), y.ctypes.data_as(D), 57, 5, 0.3, 1.0 / 57, 2.0, 0, 0.1,
                            d1.ctypes.data_as(D), R1.ctypes.data_as(D))
    assert rc == 0
    d2, R2 = oracle.q_diag_all(X, y, 0.3, 2.0)
    np.testing.assert_allclose(R1, R2, rtol=1e-13)
    np.testing.assert_allclose(d1, d2, rtol=1e-13)


def test_q_diag_tilemax_pass():
    """The one-pass diagonal, row sums and tile maxima: R and the diagonal
    equal the all-row pass; every tile maximum equals the largest |K_ij +
    lambda^2| of its pairs computed from scipy's pairwise distances (strict
    upper triangle on diagonal tiles), on a ragged size and two block edges;
    and thresholding them reproduces build_q_tile_sparse's kept tiles."""
    from scipy.spatial.distance import cdist
    p = workloads.clustered_mixture(333, 6, seed=14, gamma=0.4)
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    lam = 1.0 / p.n
    A = np.abs(np.exp(-p.gamma * cdist(X, X, "sqeuclidean")) + lam * lam)
    d0, R0 = oracle.q_diag_all(X, y, p.gamma, p.C)
    for block in (128, 50):
        d, R, tmax = oracle.q_diag_tilemax(X, y, p.gamma, p.C, block=block)
        np.testing.assert_allclose(R, R0, rtol=1e-13)
        np.testing.assert_allclose(d, d0, rtol=1e-13)
        nt = (p.n + block - 1) // block
        assert tmax.shape == (nt, nt)
        for I in range(nt):
            for J in range(nt):
                B = A[I * block:(I + 1) * block, J * block:(J + 1) * block]
                if I == J:
                    B = np.triu(B, 1)
                want = B.max() if (I <= J and B.size) else 0.0
                assert tmax[I, J] == pytest.approx(want, rel=1e-13, abs=1e-300), (block, I, J)
    _, keep = oracle.build_q_tile_sparse(X, y, p.gamma, p.C, tau=1e-3)
    _, _, tmax = oracle.q_diag_tilemax(X, y, p.gamma, p.C)
    nt = keep.shape[0]
    for I in range(nt):
        for J in range(I, nt):
            assert keep[I, J] == (I == J or tmax[I, J] > 1e-3)


def test_rows_tile_sparse_against_whole_matrix():
    """The chosen-rows pass equals the whole-matrix passes on those rows: tile
    maxima of the row's block row (both triangles, from q_diag_tilemax's
    upper triangle), whole-row |Q| sums and diagonal (q_diag_all), and the
    residual 1 - Q mu of the dense tile-sparse matrix (ragged n, two block
    edges, rows on first, inner and last blocks)."""
    p = workloads.clustered_mixture(301, 5, seed=15, gamma=0.4)
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    mu = np.random.default_rng(17).standard_normal(p.n)
    d0, R0 = oracle.q_diag_all(X, y, p.gamma, p.C)
    rows = np.array([0, 5, 127, 128, 200, 300])
    for block, tau in ((128, 1e-3), (40, 1e-2)):
        Q, keep = oracle.build_q_tile_sparse(X, y, p.gamma, p.C, tau, block=block)
        _, _, tmax_up = oracle.q_diag_tilemax(X, y, p.gamma, p.C, block=block)
        full = np.maximum(tmax_up, tmax_up.T)   # tile (I, J) and (J, I) hold the same entries
        tmax, R, d, r = oracle.rows_tile_sparse(X, y, p.gamma, p.C, tau, rows, mu, block=block)
        for k, i in enumerate(rows):
            I = i // block
            np.testing.assert_allclose(tmax[k], full[I], rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(R, R0[rows], rtol=1e-12)
        np.testing.assert_allclose(d, d0[rows], rtol=1e-12)
        want = (1.0 - Q @ mu)[rows]
        np.testing.assert_allclose(r, want, rtol=1e-11, atol=1e-12 * np.max(np.abs(want)))
        assert not keep.all()


def test_residual_tile_sparse_against_dense_matrix():
    """The kept-tiles-only residual equals 1 - Q mu with the dense tile-sparse
    matrix of build_q_tile_sparse (ragged n, two block edges)."""
    p = workloads.clustered_mixture(301, 5, seed=15, gamma=0.4)
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    mu = np.random.default_rng(16).standard_normal(p.n)
    for block, tau in ((128, 1e-3), (40, 1e-2)):
        Q, keep = oracle.build_q_tile_sparse(X, y, p.gamma, p.C, tau, block=block)
        r, rinf = oracle.residual_tile_sparse(X, y, p.gamma, np.diag(Q), keep, mu, block=block)
        want = 1.0 - Q @ mu
        np.testing.assert_allclose(r, want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))
        assert rinf == pytest.approx(np.max(np.abs(want)), rel=1e-12)
        assert not keep.all()
