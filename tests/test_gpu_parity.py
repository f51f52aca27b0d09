"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bars
* alpha: |alpha_gpu - alpha_oracle|_inf <= 1e-4 * C (the stated FP32 bar),
  and identical support-vector sets (indices whose oracle mean lies within
  SV_BAND of the threshold 0 are excluded and counted; expected 0).
* means: relative ||mu_gpu - mu_oracle||_inf / ||mu_oracle||_inf <= REL_MU.
  REL_MU = 2e-5 comes from the arithmetic: Q entries carry a relative error
  of about 1e-6 (FP32 Gram by norm expansion, expf), messages and aggregates
  are FP32 (unit roundoff 6e-8) with FP64 cross-tile sums, and the dominant
  diagonal makes every round a contraction (ratio about 1/(1 + delta)), so
  per-round errors do not grow beyond a small multiple of the Q error.
* Q entries: relative to max |Q| at 1e-5 (FP32 norm expansion vs FP64
  direct differences).
Shapes span several tiles, ragged tails (n not a multiple of 128), the
2-node case and m = 1.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu

REL_MU = 2e-5
REL_Q = 1e-5
SV_BAND_REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()
    gabp.load()


def _solve_both(p, iters, tol=0.0, **opts):
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, **opts)
    alpha, rinf, k = s.solve(iters, tol)
    mu = s.mean()
    diag_rule = opts.get("diag_rule", 0)
    Q, r = oracle.solve_svm(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C,
                            iters=iters, tol=tol, diag_rule=diag_rule)
    return s, alpha, mu, rinf, k, Q, r


def _assert_parity(p, alpha, mu, r):
    mu_o = r.mu
    rel = np.max(np.abs(mu.astype(np.float64) - mu_o)) / np.max(np.abs(mu_o))
    assert rel <= REL_MU, f"relative mean error {rel:.3e}"
    a_o = r.alpha(p.C)
    assert np.max(np.abs(alpha.astype(np.float64) - a_o)) <= 1e-4 * p.C
    band = SV_BAND_REL * np.max(np.abs(mu_o))
    clear = np.abs(mu_o) > band
    assert np.array_equal((alpha > 0)[clear], (a_o > 0)[clear])
    return rel, int((~clear).sum())


SHAPES = [(2, 3), (3, 1), (17, 7), (129, 7), (300, 64), (1000, 10)]


@pytest.mark.parametrize("n,m", SHAPES)
def test_q_formation_matches_oracle(n, m):
    p = workloads.mixture(n, m, seed=n + m, C=2.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    Qg = gabp.svm_get_q(s.h, n).astype(np.float64)
    Qo = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    err = np.max(np.abs(Qg - Qo)) / np.max(np.abs(Qo))
    assert err <= REL_Q, err
    assert np.array_equal(Qg, Qg.T)


@pytest.mark.parametrize("n,lam", [(2, 0.0), (300, 30.0), (1000, 1e3), (2500, None)])
def test_diagonal_rule_across_bias_scales(n, lam):
    """The dominant rule's row sums R_i (Section 3.1's diagonal weighting) are
    added in fixed point with a shift chosen from n and lambda^2; across bias
    scales from 0 to lambda^2 = 1e6 the diagonal must match the oracle's FP64
    sums of the whole row, relative to the diagonal, at the entries' FP32 bar."""
    p = workloads.mixture(n, 7, seed=61 + n, C=1.0)
    kw = {} if lam is None else dict(bias_mode=1, bias_lambda=lam)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, **kw)
    Qg = gabp.svm_get_q(s.h, n).astype(np.float64)
    Qo = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C, lam=lam)
    np.testing.assert_allclose(np.diag(Qg), np.diag(Qo), rtol=REL_Q)


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("iters", [0, 1, 2, 10])
def test_rounds_match_oracle(n, m, iters):
    p = workloads.mixture(n, m, seed=3 * n + m, C=1.0)
    s, alpha, mu, rinf, k, Q, r = _solve_both(p, iters)
    assert k == iters and r.kstar == iters
    _assert_parity(p, alpha, mu, r)
    # FP64 residual reported by the GPU vs the oracle's residual of the GPU means
    r_o = np.max(np.abs(1.0 - Q @ mu.astype(np.float64)))
    assert rinf == pytest.approx(r_o, rel=1e-3, abs=1e-6 * np.max(np.abs(np.diag(Q))) * np.max(np.abs(mu)))


def test_two_nodes_exact_after_one_round():
    """n = 2 is a tree: one round gives Q^-1 1 exactly (Section 2)."""
    p = workloads.mixture(2, 3, seed=5, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    Qg = gabp.svm_get_q(s.h, 2).astype(np.float64)
    for it in (1, 2, 5):
        s.refit(p.X, p.y, p.gamma, p.C)
        s.solve(it, 0.0)
        np.testing.assert_allclose(s.mean(), np.linalg.solve(Qg, np.ones(2)), rtol=2e-7)


def test_plain_small_workload_to_tolerance():
    """n=1000, m=10 FP64 two-Gaussian set: ||r||_inf < 1e-6 or 200 rounds."""
    p = workloads.plain_small()
    s, alpha, mu, rinf, k, Q, r = _solve_both(p, 200, tol=1e-6)
    assert abs(k - r.kstar) <= 1, (k, r.kstar)
    _, band = _assert_parity(p, alpha, mu, r)
    assert band == 0   # no oracle mean within the band: identical support-vector sets on every node
    st = s.stats()
    assert st["converged"] == 1 and rinf < 1e-6   # a converged solve reports residual_inf < tol
    a_o = r.alpha(p.C)
    assert st["dual_objective"] == pytest.approx(oracle.dual_objective(Q, alpha.astype(np.float64)), rel=1e-6)
    assert st["n_support"] == int((a_o > 0).sum())
    np.testing.assert_array_equal(s.support(), np.nonzero(alpha > 0)[0])


def _far_point(p, t=95.0):
    """p with its last point moved so that gamma ||x_last - x_j||^2 is about t
    for every other j: exp(-t) then lies below the smallest normal FP32 value
    (for t between about 87.3 and 103.3) while staying nonzero."""
    X = p.X.copy()
    u = np.zeros(X.shape[1], dtype=np.float32)
    u[0] = 1.0
    c = np.sqrt(max(t / p.gamma - float(np.mean(np.sum(X[:-1] ** 2, axis=1))), 1.0))
    X[-1] = c * u
    return workloads.Problem(X, p.y, p.gamma, p.C)


@pytest.mark.parametrize("task", ["svm_no_bias", "krr"])
def test_subnormal_entries_past_the_p_freeze(task):
    """Kernel entries that underflow to subnormal FP32 values (no bias term:
    the SVM with lambda = 0, and kernel ridge regression) through the rounds
    after the P messages froze (a few rounds in), against the oracle."""
    p = _far_point(workloads.mixture(300, 16, seed=21, C=1.0))
    X64 = p.X.astype(np.float64)
    d2 = np.sum((X64[:-1] - X64[-1]) ** 2, axis=1)
    k32 = np.exp(-p.gamma * d2).astype(np.float32)
    assert int(np.sum((k32 != 0) & (np.abs(k32) < np.finfo(np.float32).tiny))) > 100
    iters = 40
    if task == "krr":
        t = workloads.krr_targets(p, 3)
        s = gabp.GabpSVM(p.X, t, p.gamma, 1.0, task=gabp.TASK_KRR)
        _, r = oracle.solve_krr(p.X.astype(np.float64), t.astype(np.float64), p.gamma, 1.0, iters=iters, tol=0.0)
    else:
        s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, bias_mode=1, bias_lambda=0.0)
        _, r = oracle.solve_svm(X64, p.y.astype(np.float64), p.gamma, p.C, iters=iters, tol=0.0, lam=0.0)
    _, rinf, k = s.solve(iters, 0.0)
    mu = s.mean().astype(np.float64)
    assert k == iters and np.all(np.isfinite(mu))
    rel = np.max(np.abs(mu - r.mu)) / np.max(np.abs(r.mu))
    assert rel <= REL_MU, rel


def test_decision_matches_oracle():
    p = workloads.mixture(700, 16, seed=11, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    alpha, _, _ = s.solve(30, 0.0)
    Xt = workloads.test_points(p, 333, seed=12)
    f = s.decision(Xt).astype(np.float64)
    fo = oracle.decision(p.X.astype(np.float64), p.y.astype(np.float64), alpha.astype(np.float64),
                         Xt.astype(np.float64), p.gamma)
    assert np.max(np.abs(f - fo)) <= 1e-5 * np.max(np.abs(fo))


def test_resume_equals_one_call_and_refit_equals_create():
    p = workloads.mixture(400, 20, seed=13, C=1.0)
    s1 = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    s1.solve(7, 0.0)
    a1, _, k1 = s1.solve(5, 0.0)
    s2 = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    a2, _, k2 = s2.solve(12, 0.0)
    assert k1 == 5 and k2 == 12
    np.testing.assert_array_equal(a1, a2)
    q = workloads.mixture(400, 20, seed=14, C=3.0)
    s2.refit(q.X, q.y, q.gamma, q.C)
    a3, _, _ = s2.solve(12, 0.0)
    s3 = gabp.GabpSVM(q.X, q.y, q.gamma, q.C)
    a4, _, _ = s3.solve(12, 0.0)
    np.testing.assert_array_equal(a3, a4)


def test_device_pointer_mode_matches_host_mode():
    torch = pytest.importorskip("torch")
    p = workloads.mixture(333, 9, seed=15, C=1.0)
    sh = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    ah, _, _ = sh.solve(9, 0.0)
    Xd = torch.from_numpy(p.X).cuda()
    yd = torch.from_numpy(p.y).cuda()
    sd = gabp.GabpSVM(Xd, yd, p.gamma, p.C)
    ad, _, _ = sd.solve(9, 0.0)
    np.testing.assert_array_equal(ah, ad.cpu().numpy())
    Xt = workloads.test_points(p, 50, seed=16)
    np.testing.assert_array_equal(sh.decision(Xt), sd.decision(torch.from_numpy(Xt).cuda()).cpu().numpy())


def test_soft2_rule_failure_matches_oracle():
    """Without the dominant diagonal the dense RBF matrix leaves GaBP's
    convergence conditions: the oracle and the GPU must agree on the outcome
    (a nonpositive cavity precision, or no convergence)."""
    p = workloads.two_gaussians(200, 5, seed=17)
    try:
        oracle.solve_svm(p.X, p.y, p.gamma, p.C, iters=50, tol=1e-6, diag_rule=oracle.DIAG_SOFT2)
        oracle_failed = False
    except oracle.OracleError:
        oracle_failed = True
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, diag_rule=gabp.DIAG_SOFT2)
    if oracle_failed:
        with pytest.raises(gabp.GabpError) as ei:
            s.solve(50, 1e-6)
        assert ei.value.status == gabp.ENUMERIC
        with pytest.raises(gabp.GabpError) as ei:
            s.solve(1, 0.0)
        assert ei.value.status == gabp.ESTATE
    else:
        s.solve(50, 1e-6)


def test_invalid_inputs_rejected_on_device():
    p = workloads.mixture(64, 4, seed=18)
    X = p.X.copy()
    X[5, 2] = np.nan
    with pytest.raises(gabp.GabpError) as ei:
        gabp.GabpSVM(X, p.y, p.gamma, p.C)
    assert ei.value.status == gabp.EINVAL
    y = p.y.copy()
    y[3] = 0.5
    with pytest.raises(gabp.GabpError) as ei:
        gabp.GabpSVM(p.X, y, p.gamma, p.C)
    assert ei.value.status == gabp.EINVAL


def test_rhs_scaling_and_determinism():
    p = workloads.mixture(260, 12, seed=19)
    a = [gabp.GabpSVM(p.X, p.y, p.gamma, p.C).solve(15, 0.0)[0] for _ in range(2)]
    np.testing.assert_array_equal(a[0], a[1])


def test_p_messages_freeze_at_their_fixed_point():
    """The P recursion does not depend on b: once a round leaves every P
    message unchanged, later rounds stop writing P.  Afterwards one more round
    keeps P bitwise and updates H exactly as the oracle's single-pair update
    says."""
    p = workloads.mixture(700, 12, seed=21, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    gabp.svm_set_profiling(s.h, True)
    s.solve(120, 0.0)
    prof = gabp.svm_get_profile(s.h)
    assert prof["sweep_launches_p_frozen"] > 0, prof
    Pt0, ht0, _ = gabp.svm_get_aggregates(s.h, p.n)
    rng = np.random.default_rng(22)
    i = rng.integers(0, p.n - 1, 300)
    j = rng.integers(i + 1, p.n)
    m0 = gabp.svm_get_pairs(s.h, i, j)
    s.solve(1, 0.0)
    m1 = gabp.svm_get_pairs(s.h, i, j)
    np.testing.assert_array_equal(m1[:, :2], m0[:, :2])          # P unchanged
    X, y = p.X.astype(np.float64), p.y.astype(np.float64)
    for k in range(len(i)):
        q = oracle.q_offdiag(X[i[k]], X[j[k]], y[i[k]], y[j[k]], p.gamma, 1.0 / p.n)
        want = oracle.pair_update(q, Pt0[i[k]], ht0[i[k]], Pt0[j[k]], ht0[j[k]], m0[k].astype(np.float64))
        np.testing.assert_allclose(m1[k], want, rtol=2e-5, atol=1e-9 * np.max(np.abs(want)))
