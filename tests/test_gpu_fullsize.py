"""Parity at the full size of the benchmark workload, in the launch
configuration bench.py times (device pointers, one captured graph of 100
rounds): n=20000, m=128 FP32 mixture, gamma=1/128, C=10.

* whole solve: alpha after 100 rounds against the FP64 oracle run for the same
  100 rounds on the host (about a minute on 16 cores, 10 GB of host memory);
* one round, pair by pair: for sampled pairs, the messages the GPU writes in
  round t -> t+1 against the oracle's single-pair update computed from the
  GPU's own messages and aggregates of round t;
* aggregates: Ptilde of sampled nodes against Q_ii + sum of the incoming
  messages read back from the GPU.
"""
import os

import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu


def _mem_gb():
    for ln in open("/proc/meminfo"):
        if ln.startswith("MemAvailable:"):
            return int(ln.split()[1]) / 1e6
    return 0.0


@pytest.fixture(scope="module")
def big():
    torch = pytest.importorskip("torch")
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()
    p = workloads.plain_large()
    Xd = torch.from_numpy(p.X).cuda()
    yd = torch.from_numpy(p.y).cuda()
    h = gabp.svm_create(Xd, yd, p.gamma, p.C, gabp.opts_default(chunk=100))
    yield p, h, torch
    gabp.svm_destroy(h)


def test_full_size_solve_matches_oracle(big):
    p, h, torch = big
    if _mem_gb() < 16:
        pytest.skip("host has less than 16 GB free for the FP64 oracle")
    gabp.svm_refit(h, torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda(), p.gamma, p.C)
    alpha = torch.empty(p.n, device="cuda")
    rinf, k = gabp.svm_solve(h, 100, 0.0, alpha)
    assert k == 100
    mu = np.empty(p.n, np.float32)
    gabp.svm_get_mean(h, mu)
    Q, r = oracle.solve_svm(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C,
                            iters=100, tol=0.0)
    a = alpha.cpu().numpy().astype(np.float64)
    rel = np.max(np.abs(mu - r.mu)) / np.max(np.abs(r.mu))
    assert rel <= 2e-5, rel
    assert np.max(np.abs(a - r.alpha(p.C))) <= 1e-4 * p.C
    clear = np.abs(r.mu) > 1e-5 * np.max(np.abs(r.mu))
    assert clear.all()   # no oracle mean near the threshold: the sets are compared on every node
    assert np.array_equal(a > 0, r.alpha(p.C) > 0)
    assert rinf == pytest.approx(np.max(np.abs(1.0 - Q @ mu.astype(np.float64))), rel=1e-2, abs=1e-6)


def test_full_size_single_round_pairs_and_aggregates(big):
    p, h, torch = big
    gabp.svm_refit(h, torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda(), p.gamma, p.C)
    alpha = torch.empty(p.n, device="cuda")
    gabp.svm_solve(h, 7, 0.0, alpha)
    Pt0, ht0, _ = gabp.svm_get_aggregates(h, p.n)
    rng = np.random.default_rng(5)
    i = rng.integers(0, p.n - 1, 400)
    j = rng.integers(i + 1, p.n)
    # include diagonal-tile and last-tile pairs
    i = np.concatenate([i, [0, 5, 19968, 19990]])
    j = np.concatenate([j, [1, 127, 19999, 19999]])
    m0 = gabp.svm_get_pairs(h, i, j).astype(np.float64)
    gabp.svm_solve(h, 1, 0.0, alpha)
    m1 = gabp.svm_get_pairs(h, i, j).astype(np.float64)
    X = p.X.astype(np.float64)
    y = p.y.astype(np.float64)
    lam = 1.0 / p.n
    for k in range(len(i)):
        q = oracle.q_offdiag(X[i[k]], X[j[k]], y[i[k]], y[j[k]], p.gamma, lam)
        want = oracle.pair_update(q, Pt0[i[k]], ht0[i[k]], Pt0[j[k]], ht0[j[k]], m0[k])
        np.testing.assert_allclose(m1[k], want, rtol=2e-5, atol=1e-9 * np.max(np.abs(want)))
    # aggregates of round 8 from the messages read back
    Pt1, ht1, mu1 = gabp.svm_get_aggregates(h, p.n)
    for x in (0, 12345, 19999):
        others = np.delete(np.arange(p.n), x)
        lo, hi = np.minimum(others, x), np.maximum(others, x)
        msgs = gabp.svm_get_pairs(h, lo, hi).astype(np.float64)
        # message into x: P_ji when x is the row (x < other), P_ij when x is the column
        into_P = np.where(lo == x, msgs[:, 1], msgs[:, 0])
        into_H = np.where(lo == x, msgs[:, 3], msgs[:, 2])
        row = oracle.q_row(X, y, x, p.gamma, p.C)
        assert Pt1[x] == pytest.approx(row[x] + into_P.sum(), rel=5e-6)
        assert ht1[x] == pytest.approx(1.0 + into_H.sum(), rel=2e-5, abs=1e-6)
