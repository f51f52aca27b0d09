"""Precision form: BF16 tensor-core Gram (tcgen05) and Q stored in BF16, with
defect-correction refinement on the FP32 Gram residual.

* Q entries against the oracle fed the same BF16-rounded features: the GPU's
  FP32-accumulated BF16 Gram, rounded to BF16 for storage, is within one BF16
  rounding (2^-8 relative) of the exact entry; the weighted diagonal comes
  from the accurate (unrounded) matrix.
* an unrefined BF16 solve against the oracle run on the same BF16 matrix.
* a refined solve against the oracle's fixed point of the exact FP64 matrix
  (FP64 Cholesky), at the FP32 bars: |dalpha|_inf <= 1e-4 C, relative mean
  error <= 2e-5, identical support vectors.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()


def _bf16_matrix(p):
    """The matrix the BF16 sweeps see: off-diagonal from BF16 features, rounded
    to BF16; diagonal from the exact matrix of the FP32 features."""
    X = p.X.astype(np.float64)
    y = p.y.astype(np.float64)
    Qx = oracle.build_q(X, y, p.gamma, p.C)
    Qb = bf16(oracle.build_q(bf16(p.X), y, p.gamma, p.C))
    Qb[np.diag_indices(p.n)] = np.diag(Qx)
    return Qx, Qb


@pytest.mark.parametrize("n,m", [(129, 7), (300, 64), (520, 100)])
def test_bf16_q_formation(n, m):
    p = workloads.mixture(n, m, seed=40 + n, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16)
    Qg = gabp.svm_get_q(s.h, n).astype(np.float64)
    Qx, Qb = _bf16_matrix(p)
    off = ~np.eye(n, dtype=bool)
    exact_bf = oracle.build_q(bf16(p.X), p.y.astype(np.float64), p.gamma, p.C)
    err = np.abs(Qg - exact_bf)[off]
    assert np.all(err <= 2.0 ** -8 * np.abs(exact_bf[off]) + 1e-6 * np.max(np.abs(exact_bf))), err.max()
    np.testing.assert_allclose(np.diag(Qg), np.diag(Qx), rtol=1e-5)
    # most entries round identically
    assert np.mean(Qg[off] == Qb[off]) > 0.95


# Entries of the GPU's BF16 matrix that differ from the independently rounded
# oracle matrix (by one BF16 unit: the FP32 value lies near a rounding
# boundary) are at most this fraction of all entries (asserted by the
# formation test above).
F_DISAGREE = 0.05


def _bf16_tolerance(Qb, mu_ref):
    """Relative max-norm tolerance between a BF16-matrix solve on the GPU and
    the oracle's on Qb, derived from the one-unit disagreements: entry (i, j)
    differs with probability at most F_DISAGREE, by at most one BF16 unit
    (2^-8 |Q_ij| relative, either sign), so (dQ mu)_i has a standard deviation
    of at most 2^-8 sqrt(F_DISAGREE sum_j (Q_ij mu_j)^2), and the dominant
    diagonal passes it to mu_i divided by about Q_ii.  Six standard
    deviations, plus the FP32 arithmetic bar 2e-5."""
    off = Qb - np.diag(np.diag(Qb))
    sd = 2.0 ** -8 * np.sqrt(F_DISAGREE * ((off * mu_ref[None, :]) ** 2).sum(axis=1)) / np.diag(Qb)
    return 6.0 * float(sd.max()) / float(np.max(np.abs(mu_ref))) + 2e-5


@pytest.mark.parametrize("n,m", [(300, 64), (1000, 10)])
def test_bf16_solve_matches_oracle_on_bf16_matrix(n, m):
    """Unrefined BF16 solves against the oracle run on the independently
    rounded BF16 matrix Qb: 12 rounds (iterates) and to convergence (the
    fixed point Qb^-1 1), within the tolerance derived above."""
    p = workloads.mixture(n, m, seed=50 + n, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16)
    alpha, rinf, k = s.solve(12, 0.0)
    mu = s.mean().astype(np.float64)
    _, Qb = _bf16_matrix(p)
    ref = np.linalg.solve(Qb, np.ones(n))
    tol = _bf16_tolerance(Qb, ref)
    assert tol < 5e-4, tol
    r2 = oracle.gabp(Qb, np.ones(n), iters=12)
    assert np.max(np.abs(mu - r2.mu)) / np.max(np.abs(r2.mu)) <= tol
    s.refit(p.X, p.y, p.gamma, p.C)
    s.solve(400, 1e-6)
    mu = s.mean().astype(np.float64)
    assert s.stats()["converged"] == 1
    # stopped at an in-sweep residual below 1e-6 on the BF16 matrix: Varah's
    # bound adds 1e-6 / min_i (Qb_ii - sum_j |Qb_ij|) to the distance from ref
    margin = float(np.min(2 * np.diag(Qb) - np.abs(Qb).sum(axis=1)))
    assert margin > 0
    slack = 1e-6 / margin / np.max(np.abs(ref))
    assert np.max(np.abs(mu - ref)) / np.max(np.abs(ref)) <= tol + slack


@pytest.mark.parametrize("n,m,C", [(300, 64, 1.0), (1000, 10, 1.0), (777, 33, 10.0)])
def test_refined_solve_reaches_fp64_fixed_point(n, m, C):
    p = workloads.mixture(n, m, seed=60 + n, C=C)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16, refine=8)
    alpha, rinf, k = s.solve(200, 1e-6)
    st = s.stats()
    mu = s.mean().astype(np.float64)
    Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    ref = np.linalg.solve(Qx, np.ones(n))
    rel = np.max(np.abs(mu - ref)) / np.max(np.abs(ref))
    assert rel <= 2e-5, (rel, st)
    a_ref = np.clip(ref, 0, p.C)
    assert np.max(np.abs(alpha.astype(np.float64) - a_ref)) <= 1e-4 * p.C
    clear = np.abs(ref) > 1e-5 * np.max(np.abs(ref))
    assert np.array_equal((alpha > 0)[clear], (a_ref > 0)[clear])
    assert st["refine_passes"] >= 1 and rinf < 1e-6
    # the FP64 residual of the GPU answer, by the oracle, agrees
    assert np.max(np.abs(1.0 - Qx @ mu)) < 2e-6


@pytest.mark.parametrize("n,m", [(129, 7), (300, 64), (700, 100)])
def test_recompute_equals_bf16_store(n, m):
    """Recomputing the BF16 Q tiles inside every sweep gives exactly the
    values the BF16 store holds, so both forms agree bitwise."""
    p = workloads.mixture(n, m, seed=70 + n, C=1.0)
    a_store, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16).solve(9, 0.0)
    s_rc = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_RECOMPUTE)
    a_rc, _, k = s_rc.solve(9, 0.0)
    assert k == 9
    np.testing.assert_array_equal(a_store, a_rc)
    with pytest.raises(gabp.GabpError):
        gabp.svm_get_q(s_rc.h, n)


def test_refined_recompute_reaches_fp64_fixed_point():
    p = workloads.mixture(900, 64, seed=81, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_RECOMPUTE, refine=8)
    alpha, rinf, k = s.solve(200, 1e-6)
    mu = s.mean().astype(np.float64)
    Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    ref = np.linalg.solve(Qx, np.ones(p.n))
    assert np.max(np.abs(mu - ref)) / np.max(np.abs(ref)) <= 2e-5
    assert np.max(np.abs(alpha.astype(np.float64) - np.clip(ref, 0, p.C))) <= 1e-4 * p.C
    assert rinf < 1e-6


@pytest.mark.parametrize("q_mode", [gabp.Q_BF16, gabp.Q_RECOMPUTE])
@pytest.mark.parametrize("n,m,C", [(300, 64, 1.0), (1000, 10, 1.0), (777, 33, 10.0)])
def test_bf16_messages_refined_reach_fp64_fixed_point(q_mode, n, m, C):
    """Messages stored in BF16 (arithmetic FP32): the rounding error of the
    stored messages is removed by the defect correction on the FP32-Gram
    residual, so the answer meets the same FP32 bars as the plain form."""
    p = workloads.mixture(n, m, seed=90 + n, C=C)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=q_mode, refine=10, msg_bf16=1)
    alpha, rinf, k = s.solve(300, 1e-6)
    mu = s.mean().astype(np.float64)
    Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    ref = np.linalg.solve(Qx, np.ones(p.n))
    assert np.max(np.abs(mu - ref)) / np.max(np.abs(ref)) <= 2e-5
    a_ref = np.clip(ref, 0, p.C)
    assert np.max(np.abs(alpha.astype(np.float64) - a_ref)) <= 1e-4 * p.C
    clear = np.abs(ref) > 1e-5 * np.max(np.abs(ref))
    assert np.array_equal((alpha > 0)[clear], (a_ref > 0)[clear])
    assert rinf < 1e-6 and s.stats()["converged"] == 1


def test_bf16_messages_rejected_for_plain_form():
    p = workloads.mixture(50, 3, seed=99)
    with pytest.raises(gabp.GabpError) as ei:
        gabp.GabpSVM(p.X, p.y, p.gamma, p.C, msg_bf16=1)
    assert ei.value.status == gabp.EINVAL


@pytest.mark.parametrize("handover,inner", [(1e-2, 1e-2), (1e-5, 3e-3)])
def test_refinement_schedule_options_keep_the_bars(handover, inner):
    """The refinement thresholds are options; any schedule still ends at the
    FP64 fixed point within the FP32 bars (only the round count changes)."""
    p = workloads.mixture(600, 24, seed=95, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, q_mode=gabp.Q_BF16, refine=12, msg_bf16=1,
                     refine_handover=handover, refine_inner=inner)
    alpha, rinf, k = s.solve(400, 1e-6)
    Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
    ref = np.linalg.solve(Qx, np.ones(p.n))
    mu = s.mean().astype(np.float64)
    assert np.max(np.abs(mu - ref)) / np.max(np.abs(ref)) <= 2e-5
    assert np.max(np.abs(alpha.astype(np.float64) - np.clip(ref, 0, p.C))) <= 1e-4 * p.C
    assert rinf < 1e-6 and s.stats()["converged"] == 1
