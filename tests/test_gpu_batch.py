"""Batched and served forms against the single-instance solver and the oracle.

* every instance of a batch (uneven n, m, C, gamma; one persistent launch per
  round for all of them) gives the same alpha as solving it alone, and
  matches the FP64 oracle at the FP32 bars;
* per-instance stop tests: instances converge after different numbers of
  rounds, each at its own first round with ||r||_inf < tol;
* the precision form (BF16 tensor-core Q + refinement) reaches the FP64
  fixed point in the batch;
* the server: requests admitted over several steps (continuous batching)
  give the same results as alone.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(130, 700))
        m = int(rng.choice([8, 32, 128]))
        C = float(rng.choice([0.1, 1.0, 10.0]))
        g = float(rng.choice([0.5, 1.0, 2.0])) / m
        p = workloads.mixture(n, m, seed=seed * 100 + k, gamma=g, C=C)
        out.append(p)
    return out


def test_batch_equals_single_and_oracle():
    probs = _mix(10, 1)
    alphas, res, rc = gabp.batch_solve(probs, 25, 0.0, chunk=8)
    assert rc == gabp.OK
    for p, a, r in zip(probs, alphas, res):
        assert r["status"] == 0 and r["iters_done"] == 25
        single, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C).solve(25, 0.0)
        np.testing.assert_array_equal(a, single)
        _, ro = oracle.solve_svm(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C, iters=25)
        assert np.max(np.abs(a - ro.alpha(p.C))) <= 1e-4 * p.C
        assert np.max(np.abs(ro.mu)) > 0


def test_batch_per_instance_convergence_and_autotune():
    probs = _mix(8, 2)
    alphas, res, rc = gabp.batch_solve(probs, 300, 1e-6, chunk=0)
    assert rc == gabp.OK
    ks = []
    for p, a, r in zip(probs, alphas, res):
        # the stop test (in-sweep residual, compensated FP32 sums) and the final
        # FP32-Gram / FP64 residual sum the same terms in different orders
        assert r["converged"] == 1 and r["residual_inf"] < 1e-6
        _, ro = oracle.solve_svm(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C,
                                 iters=300, tol=1e-6)
        ks.append(ro.kstar)
        assert abs(r["iters_done"] - (ro.kstar + 1)) <= 1, (r["iters_done"], ro.kstar)
        assert np.max(np.abs(a - ro.alpha(p.C))) <= 1e-4 * p.C
    assert len(set(ks)) > 1      # the instances did stop at different rounds


def test_batch_precision_form_refined():
    probs = _mix(6, 3)
    alphas, res, rc = gabp.batch_solve(probs, 300, 1e-6, chunk=8, q_mode=gabp.Q_BF16, refine=8)
    assert rc == gabp.OK
    for p, a, r in zip(probs, alphas, res):
        Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
        ref = np.linalg.solve(Qx, np.ones(p.n))
        assert r["residual_inf"] < 1e-6 and r["refine_passes"] >= 1
        assert np.max(np.abs(a - np.clip(ref, 0, p.C))) <= 1e-4 * p.C


def test_server_results_equal_alone():
    probs = _mix(9, 4)
    srv = gabp.Server(iters=300, tol=1e-6, max_members=4, chunk=4)
    tickets = []
    # arrivals spread over steps: 3 now, then 2 per step
    for p in probs[:3]:
        tickets.append(srv.submit(p.X, p.y, p.gamma, p.C))
    pending = list(probs[3:])
    out = {}
    for _ in range(2000):
        if pending:
            for p in pending[:2]:
                tickets.append(srv.submit(p.X, p.y, p.gamma, p.C))
            pending = pending[2:]
        active, queued, done = srv.step()
        assert active <= 4
        fresh = srv.completed()
        new = []
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
                    new.append(t)
        assert sorted(fresh) == sorted(new)   # completed() reports exactly the newly finished
        if len(out) == len(probs) and not pending:
            break
    assert len(out) == len(probs)
    assert srv.completed() == []
    for t, p in zip(tickets, probs):
        a, r = out[t]
        assert r["status"] == 0 and r["converged"] == 1
        single, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, chunk=4).solve(300, 1e-6)
        np.testing.assert_array_equal(a, single)
    srv.close()


def test_batch_bf16_messages_refined():
    probs = _mix(6, 5)
    alphas, res, rc = gabp.batch_solve(probs, 300, 1e-6, chunk=8, q_mode=gabp.Q_BF16, refine=10, msg_bf16=1)
    assert rc == gabp.OK
    for p, a, r in zip(probs, alphas, res):
        Qx = oracle.build_q(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C)
        ref = np.linalg.solve(Qx, np.ones(p.n))
        assert r["residual_inf"] < 1e-6 and r["converged"] == 1
        assert np.max(np.abs(a - np.clip(ref, 0, p.C))) <= 1e-4 * p.C


def test_server_krr_and_phases():
    """The regression task through the server equals the single solve, and the
    server reports its phase times."""
    srv = gabp.Server(iters=300, tol=1e-6, max_members=3, chunk=4, task=gabp.TASK_KRR)
    probs, tickets = [], []
    for k, (n, m) in enumerate([(200, 8), (350, 16), (500, 32), (260, 8)]):
        p = workloads.mixture(n, m, seed=70 + k)
        t = workloads.krr_targets(p, 80 + k)
        probs.append((p, t))
        tickets.append(srv.submit(p.X, t, p.gamma, 0.5))
    out = {}
    for _ in range(2000):
        srv.step()
        for t in srv.completed():
            out[t] = srv.poll(t)
        if len(out) == len(tickets):
            break
    assert len(out) == len(tickets)
    ph = srv.phases()
    assert ph["steps"] >= 1 and ph["total_ms"] > 0 and ph["rounds_ms"] > 0
    assert all(ph[k] >= 0 for k in ph)
    for t, (p, tg) in zip(tickets, probs):
        a, r = out[t]
        assert r["status"] == 0 and r["converged"] == 1
        single, _, _ = gabp.GabpSVM(p.X, tg, p.gamma, 0.5, task=gabp.TASK_KRR, chunk=4).solve(300, 1e-6)
        np.testing.assert_array_equal(a, single)
    srv.close()


def test_batch_device_pointers_equal_host():
    torch = pytest.importorskip("torch")
    probs = _mix(5, 6)
    a_host, r_host, rc = gabp.batch_solve(probs, 60, 1e-6, chunk=8)
    assert rc == gabp.OK
    dprobs = [workloads.Problem(torch.from_numpy(p.X).cuda(), torch.from_numpy(p.y).cuda(), p.gamma, p.C)
              for p in probs]
    a_dev, r_dev, rc = gabp.batch_solve(dprobs, 60, 1e-6, chunk=8)
    assert rc == gabp.OK
    for ah, ad, rh, rd in zip(a_host, a_dev, r_host, r_dev):
        np.testing.assert_array_equal(ah, ad.cpu().numpy())
        assert rh["iters_done"] == rd["iters_done"]


def _grid(seeds=(31, 32), n=(300, 170), m=(32, 8)):
    """Parameter grids (C x gamma) over shared feature arrays: the instances
    of one grid pass the same X, so formation computes their Gram tiles once."""
    out = []
    for s, nn, mm in zip(seeds, n, m):
        base = workloads.mixture(nn, mm, seed=s)
        for C in (0.1, 1.0, 10.0):
            for g in (0.5, 1.0, 2.0):
                out.append(workloads.Problem(base.X, base.y, g / mm, C))
    return out


@pytest.mark.parametrize("kw", [dict(q_mode=0), dict(q_mode=1, refine=4), dict(q_mode=2, refine=4),
                                dict(q_mode=0, task=gabp.TASK_KRR)])
def test_batch_parameter_grid_shares_gram(kw):
    torch = pytest.importorskip("torch")
    grid = _grid()
    assert grid[0].X is grid[1].X
    if kw.get("task") == gabp.TASK_KRR:
        grid = [workloads.Problem(p.X, workloads.krr_targets(p, seed=5), p.gamma, p.C) for p in grid]
    # the same problems with private copies of their features (no sharing)
    private = [workloads.Problem(p.X.copy(), p.y.copy(), p.gamma, p.C) for p in grid]
    a_sh, r_sh, rc = gabp.batch_solve(grid, 40, 0.0, chunk=8, **kw)
    assert rc == gabp.OK
    a_pr, r_pr, rc = gabp.batch_solve(private, 40, 0.0, chunk=8, **kw)
    assert rc == gabp.OK
    # device arrays shared per grid, as a parameter search passes them
    dev = {}
    for p in grid:
        if id(p.X) not in dev:
            dev[id(p.X)] = (torch.from_numpy(p.X).cuda(), torch.from_numpy(np.ascontiguousarray(p.y)).cuda())
    dgrid = []
    for p in grid:
        X, y = dev[id(p.X)]
        if kw.get("task") == gabp.TASK_KRR:
            y = torch.from_numpy(np.ascontiguousarray(p.y)).cuda()
        dgrid.append(workloads.Problem(X, y, p.gamma, p.C))
    a_dv, r_dv, rc = gabp.batch_solve(dgrid, 40, 0.0, chunk=8, **kw)
    assert rc == gabp.OK
    for p, a, b, d, rs, rp in zip(grid, a_sh, a_pr, a_dv, r_sh, r_pr):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, d.cpu().numpy())
        assert rs["residual_inf"] == rp["residual_inf"] and rs["iters_done"] == rp["iters_done"]
    if kw.get("q_mode", 0) == 0:
        # and each equals its oracle iterate at the FP32 bar
        for p, a in list(zip(grid, a_sh))[::4]:
            if kw.get("task") == gabp.TASK_KRR:
                # (C is the ridge for this task)
                _, ro = oracle.solve_krr(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C, iters=40,
                                         tol=0.0)
                assert np.max(np.abs(a - ro.mu)) <= 2e-5 * np.max(np.abs(ro.mu))
            else:
                _, ro = oracle.solve_svm(p.X.astype(np.float64), p.y.astype(np.float64), p.gamma, p.C, iters=40,
                                         tol=0.0)
                assert np.max(np.abs(a - ro.alpha(p.C))) <= 1e-4 * p.C


def test_server_parameter_grid_shares_gram():
    grid = _grid(seeds=(41,), n=(260,), m=(16,))
    srv = gabp.Server(iters=60, tol=1e-6, max_members=4, chunk=4)
    tickets = [srv.submit(p.X, p.y, p.gamma, p.C) for p in grid]
    out = {}
    for _ in range(2000):
        srv.step()
        for t in srv.completed():
            out[t] = srv.poll(t)
        if len(out) == len(grid):
            break
    srv.close()
    assert len(out) == len(grid)
    for p, t in zip(grid, tickets):
        a, r = out[t]
        assert r["status"] == 0
        single, _, _ = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, chunk=4).solve(60, 1e-6)
        np.testing.assert_array_equal(a, single)


def test_batch_mixes_finalize_modes():
    """Instances with at most 32 tile rows are finalized one warp per node
    block, larger ones one CTA per block; a list holding both gives each
    instance the same result as solving it alone (synchronous and staged)."""
    probs = [workloads.mixture(300, 16, seed=61), workloads.mixture(4500, 8, seed=62),
             workloads.mixture(4097, 8, seed=63), workloads.mixture(4096, 8, seed=64)]
    for stages in (1, 3):
        alphas, res, rc = gabp.batch_solve(probs, 30, 1e-7, chunk=4, stages=stages)
        assert rc == gabp.OK
        for p, a, r in zip(probs, alphas, res):
            single, rinf, k = gabp.GabpSVM(p.X, p.y, p.gamma, p.C, chunk=4, stages=stages).solve(30, 1e-7)
            np.testing.assert_array_equal(a, single)
            assert r["iters_done"] == k
            assert r["residual_inf"] == pytest.approx(rinf, rel=1e-6)


def test_batch_engine_kept_between_calls():
    """The engine kept from one gabp_batch_solve serves the next compatible
    call (same or fewer instances) and gives the same results as a fresh one;
    other options build a new engine."""
    probs = _mix(6, 9)
    gabp.batch_release()
    a0, r0, rc = gabp.batch_solve(probs, 40, 1e-6, chunk=0)
    assert rc == gabp.OK
    a1, r1, _ = gabp.batch_solve(probs, 40, 1e-6, chunk=0)
    a2, r2, _ = gabp.batch_solve(probs[:3], 40, 1e-6, chunk=0)
    gabp.batch_solve(probs, 40, 1e-6, chunk=0, q_mode=gabp.Q_BF16, refine=4)
    a3, r3, _ = gabp.batch_solve(probs, 40, 1e-6, chunk=4)
    gabp.batch_release()
    gabp.batch_release()
    for a in (a1, a3):
        for x, y in zip(a, a0):
            np.testing.assert_array_equal(x, y)
    for x, y in zip(a2, a0[:3]):
        np.testing.assert_array_equal(x, y)
    for r in (r1, r3):
        assert [q["iters_done"] for q in r] == [q["iters_done"] for q in r0]


def _offset_copy(a, offset_bytes):
    """A C-contiguous copy of `a` whose data starts `offset_bytes` past a
    64-byte boundary (host inputs not aligned to 16 bytes)."""
    buf = np.zeros(a.nbytes + 128, dtype=np.uint8)
    start = (-buf.ctypes.data) % 64 + offset_bytes
    out = np.frombuffer(buf.data, dtype=a.dtype, count=a.size, offset=start).reshape(a.shape)
    out[...] = a
    assert out.ctypes.data % 16 == offset_bytes % 16
    return out


def test_batch_host_inputs_any_alignment():
    """Host (pageable) inputs are copied in whatever way the platform offers
    (a copy kernel where the GPU reads pageable memory, 16-byte or 4-byte
    words, else the driver's copy); misaligned buffers give the same results
    as aligned ones."""
    probs = _mix(4, 11)
    a0, r0, rc = gabp.batch_solve(probs, 30, 1e-6, chunk=4)
    assert rc == gabp.OK
    mis = [workloads.Problem(_offset_copy(p.X, 4), _offset_copy(np.asarray(p.y, np.float32), 8), p.gamma, p.C)
           for p in probs]
    a1, r1, rc = gabp.batch_solve(mis, 30, 1e-6, chunk=4)
    assert rc == gabp.OK
    for x, y in zip(a0, a1):
        np.testing.assert_array_equal(x, y)


def test_batch_grid_fp64_inputs_share_gram():
    """FP64 host features (converted on the device while the instances are
    added) shared by a grid give the same results as private copies, and as
    the FP32 rounding of the same features."""
    grid = _grid(seeds=(51,), n=(230,), m=(12,))
    g64 = [workloads.Problem(grid[0].X.astype(np.float64), p.y, p.gamma, p.C) for p in grid]
    for p in g64[1:]:
        p.X = g64[0].X
    private = [workloads.Problem(p.X.copy(), p.y, p.gamma, p.C) for p in g64]
    a_sh, _, rc = gabp.batch_solve(g64, 30, 0.0, chunk=8)
    assert rc == gabp.OK
    a_pr, _, rc = gabp.batch_solve(private, 30, 0.0, chunk=8)
    assert rc == gabp.OK
    a_32, _, rc = gabp.batch_solve(grid, 30, 0.0, chunk=8)
    assert rc == gabp.OK
    for x, y, z in zip(a_sh, a_pr, a_32):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
