"""Block Gauss-Seidel (staged) message schedule against the FP64 oracle's
staged schedule.  A round updates every pair once, in S stages over bands
of tile columns (stage bounds from the same integer rule on both sides, node
blocks of the 128-row tiles); later stages use the aggregates formed after
the earlier ones.  Bars as for the synchronous schedule: relative mean error
2e-5, |dalpha|_inf <= 1e-4 C, the stop round within one of the oracle's.
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


def _rel(a, b):
    return np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("n,m", [(300, 64), (700, 12), (1000, 10)])
@pytest.mark.parametrize("stages", [2, 4])
@pytest.mark.parametrize("iters", [1, 2, 10])
def test_staged_rounds_match_oracle(n, m, stages, iters):
    p = workloads.mixture(n, m, seed=5 * n + m, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=stages)
    alpha, rinf, k = s.solve(iters, 0.0)
    Q = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    r = oracle.gabp_staged(Q, np.ones(n), iters=iters, stages=stages, block=128)
    assert k == iters
    assert _rel(s.mean(), r.mu) <= REL
    assert np.max(np.abs(alpha.astype(np.float64) - r.alpha(p.C))) <= 1e-4 * p.C


def test_one_stage_is_the_synchronous_schedule():
    p = workloads.mixture(500, 16, seed=3)
    a0, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C).solve(20, 0.0)
    a1, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=1).solve(20, 0.0)
    np.testing.assert_array_equal(a0, a1)


@pytest.mark.parametrize("stages", [2, 4, 8])
def test_staged_to_tolerance_in_fewer_rounds(stages):
    p = workloads.mixture(1500, 24, seed=17, C=10.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=stages)
    alpha, rinf, k = s.solve(300, 1e-6)
    Q = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    r = oracle.gabp_staged(Q, np.ones(p.n), iters=300, tol=1e-6, stages=stages, block=128)
    ks = oracle.gabp(Q, np.ones(p.n), iters=300, tol=1e-6).kstar
    assert abs(k - r.kstar) <= 1 and r.kstar < ks
    assert s.stats()["converged"] == 1 and rinf < 1e-6
    assert _rel(s.mean(), r.mu) <= REL
    ref = np.linalg.solve(Q, np.ones(p.n))
    assert np.max(np.abs(alpha.astype(np.float64) - np.clip(ref, 0, p.C))) <= 1e-4 * p.C


def test_staged_with_frozen_p():
    """A long staged run: P freezes, the frozen rounds still follow the oracle."""
    p = workloads.mixture(900, 12, seed=23, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=3)
    gabp.svm_set_profiling(s.h, True)
    s.solve(80, 0.0)
    assert gabp.svm_get_profile(s.h)["sweep_launches_p_frozen"] > 0
    Q = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    r = oracle.gabp_staged(Q, np.ones(p.n), iters=80, stages=3, block=128)
    assert _rel(s.mean(), r.mu) <= REL


def test_staged_batch_equals_single():
    rng = np.random.default_rng(9)
    probs = []
    for k in range(6):
        n = int(rng.integers(130, 900))
        m = int(rng.choice([8, 32, 128]))
        probs.append(workloads.mixture(n, m, seed=200 + k, C=float(rng.choice([0.1, 1.0, 10.0]))))
    alphas, res, rc = gabp.batch_solve(probs, 200, 1e-6, chunk=8, stages=4)
    assert rc == gabp.OK
    for p, a, r in zip(probs, alphas, res):
        assert r["status"] == 0 and r["converged"] == 1
        single, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=4, chunk=8).solve(200, 1e-6)
        np.testing.assert_array_equal(a, single)


def test_staged_precision_form_refined():
    p = workloads.mixture(777, 33, seed=31, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16, refine=10, msg_bf16=1, stages=4)
    alpha, rinf, k = s.solve(300, 1e-6)
    Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    ref = np.linalg.solve(Qx, np.ones(p.n))
    assert _rel(s.mean(), ref) <= REL and rinf < 1e-6
    assert np.max(np.abs(alpha.astype(np.float64) - np.clip(ref, 0, p.C))) <= 1e-4 * p.C


def test_staged_krr():
    p = workloads.mixture(640, 20, seed=41)
    t = workloads.krr_targets(p, 42)
    s = gabp.GabpSVM(p.X, t, p.gamma, 0.5, task=gabp.TASK_KRR, stages=2)
    c, rinf, k = s.solve(12, 0.0)
    Q = oracle.build_q_krr(p.X.astype(np.float64), p.gamma, 0.5)
    r = oracle.gabp_staged(Q, t.astype(np.float64), iters=12, stages=2, block=128)
    assert _rel(c, r.mu) <= REL


def test_stages_option_validated():
    p = workloads.mixture(64, 4, seed=1)
    with pytest.raises(gabp.GabpError) as ei:
        gabp.GabpSVM(p.X, p.y, p.gamma, p.C, stages=17)
    assert ei.value.status == gabp.EINVAL
