"""Kernel ridge regression (Section 1.2) on the same sweep: the GPU path with
task = KRR against the FP64 oracle's KRR solve.

KRR solves (K + lambda_r I) c = t with real targets t: no labels in the
matrix, right-hand side t, coefficients unclipped, prediction
f(x) = sum_i c_i K(x_i, x).  Bars as for the SVM: relative mean error
2e-5 (FP32 arithmetic, contraction of the dominant diagonal), Q entries
1e-5 of max |Q|, predictions 1e-5 of max |f|.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()


def _case(n, m, seed):
    p = workloads.mixture(n, m, seed=seed)
    t = workloads.krr_targets(p, seed + 1)
    return p, t


def _rel(a, b):
    return np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("n,m", [(2, 3), (129, 7), (300, 64), (1000, 10)])
@pytest.mark.parametrize("iters", [0, 1, 10])
def test_krr_rounds_match_oracle(n, m, iters):
    p, t = _case(n, m, 3 * n + m)
    ridge = 0.5
    s = gabp.GabpSVM(p.X, t, p.gamma, ridge, task=gabp.TASK_KRR)
    c, rinf, k = s.solve(iters, 0.0)
    Q, r = oracle.solve_krr(p.X.astype(np.float64), t.astype(np.float64), p.gamma, ridge, iters=iters, tol=0.0)
    assert k == iters
    assert _rel(s.mean(), r.mu) <= REL
    np.testing.assert_array_equal(c, s.mean())          # coefficients are the unclipped means
    mu = s.mean().astype(np.float64)
    r_o = np.max(np.abs(t.astype(np.float64) - Q @ mu))
    assert rinf == pytest.approx(r_o, rel=1e-3, abs=1e-6 * np.max(np.abs(np.diag(Q))) * np.max(np.abs(mu)))
    Qg = gabp.svm_get_q(s.h, n).astype(np.float64)
    assert np.max(np.abs(Qg - Q)) / np.max(np.abs(Q)) <= 1e-5


def test_krr_ridge_solve_and_prediction():
    """soft2 rule with a diagonally dominant ridge: the converged coefficients
    are (K + ridge I)^-1 t; predictions match the oracle's."""
    p, t = _case(700, 16, 21)
    X = p.X.astype(np.float64)
    Qo = oracle.build_q_krr(X, p.gamma, 1.0, diag_rule=oracle.DIAG_SOFT2)
    ridge = 1.2 * (np.abs(Qo).sum(1) - np.diag(Qo)).max()
    s = gabp.GabpSVM(p.X, t, p.gamma, ridge, task=gabp.TASK_KRR, diag_rule=gabp.DIAG_SOFT2)
    c, rinf, k = s.solve(500, 1e-6)
    Q, r = oracle.solve_krr(X, t.astype(np.float64), p.gamma, ridge, iters=500, tol=1e-6,
                            diag_rule=oracle.DIAG_SOFT2)
    assert abs(k - r.kstar) <= 1 and rinf < 1e-6
    ref = np.linalg.solve(Q, t.astype(np.float64))
    assert _rel(c, ref) <= REL
    Xt = workloads.test_points(p, 200, seed=22)
    f = s.decision(Xt).astype(np.float64)
    fo = oracle.decision(X, np.ones(p.n), c.astype(np.float64), Xt.astype(np.float64), p.gamma, lam=0.0)
    assert np.max(np.abs(f - fo)) <= 1e-5 * np.max(np.abs(fo))
    st = s.stats()
    obj = t.astype(np.float64) @ c - 0.5 * c.astype(np.float64) @ Q @ c.astype(np.float64)
    assert st["dual_objective"] == pytest.approx(obj, rel=1e-6)
    assert st["n_support"] == int((np.abs(c) > 0).sum())


@pytest.mark.parametrize("msg_bf16", [0, 1])
def test_krr_precision_form_refined(msg_bf16):
    p, t = _case(777, 33, 31)
    s = gabp.GabpSVM(p.X, t, p.gamma, 0.5, task=gabp.TASK_KRR, q_mode=gabp.Q_BF16, refine=10, msg_bf16=msg_bf16)
    c, rinf, k = s.solve(300, 1e-6)
    Q = oracle.build_q_krr(p.X.astype(np.float64), p.gamma, 0.5)
    ref = np.linalg.solve(Q, t.astype(np.float64))
    assert _rel(c, ref) <= REL and rinf < 1e-6
    assert s.stats()["refine_passes"] >= 1


def test_krr_batch_equals_single():
    probs, targets = [], []
    for k, (n, m) in enumerate([(150, 8), (300, 32), (520, 128)]):
        p, t = _case(n, m, 40 + k)
        probs.append(workloads.Problem(p.X, t, p.gamma, 0.3 + 0.2 * k))
        targets.append(t)
    alphas, res, rc = gabp.batch_solve(probs, 200, 1e-6, chunk=8, task=gabp.TASK_KRR)
    assert rc == gabp.OK
    for p, a, r in zip(probs, alphas, res):
        assert r["status"] == 0 and r["converged"] == 1
        single, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, task=gabp.TASK_KRR, chunk=8).solve(200, 1e-6)
        np.testing.assert_array_equal(a, single)


def test_krr_targets_validated():
    p, t = _case(64, 4, 50)
    bad = t.copy()
    bad[7] = np.nan
    with pytest.raises(gabp.GabpError) as ei:
        gabp.GabpSVM(p.X, bad, p.gamma, 1.0, task=gabp.TASK_KRR)
    assert ei.value.status == gabp.EINVAL
    # real targets are fine for KRR, not for the SVM
    gabp.GabpSVM(p.X, t, p.gamma, 1.0, task=gabp.TASK_KRR)
    with pytest.raises(gabp.GabpError):
        gabp.GabpSVM(p.X, t, p.gamma, 1.0)
