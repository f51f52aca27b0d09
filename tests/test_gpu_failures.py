"""Failure detection without faulting the GPU: the bounded device-side wait
runs out on a barrier nothing completes and reports GABP_ETIMEOUT, and the
context stays usable for a solve afterwards."""
import numpy as np
import pytest

from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()
    assert gabp.selftest_bounded_wait(50_000_000) == gabp.ETIMEOUT     # 50 ms
    p = workloads.mixture(200, 5, seed=3)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    alpha, rinf, k = s.solve(30, 0.0)
    assert k == 30 and np.all(np.isfinite(alpha))


def test_sweep_reciprocal_within_one_ulp_of_ieee_division():
    """The sweep's reciprocal (hardware approximation + one Newton-Raphson
    step) against correctly rounded FP32 division, over the magnitudes cavity
    precisions take (1e-6 .. 1e8) and random mantissas."""
    rng = np.random.default_rng(5)
    d = (10.0 ** rng.uniform(-6, 8, 200000)).astype(np.float32)
    d = np.concatenate([d, np.float32([1.0, 2.0, 3.0, 0.1, 1e-6, 1e8])])
    got = gabp.selftest_reciprocal(d)
    want = (np.float32(1.0) / d).astype(np.float32)
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1, ulp.max()
    assert np.mean(ulp == 0) > 0.9


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_over_budget_create_returns_enomem_before_any_device_work():
    """A dense instance whose plan (8 n^2 bytes of messages + 2 n^2 of FP32 Q
    at n = 200000: 400 GB) exceeds the device: GABP_ENOMEM from the budget
    check, no handle, and the device's free memory unchanged."""
    p = workloads.mixture(200000, 4, seed=1)
    free0 = _free_bytes()
    with pytest.raises(gabp.GabpError) as ei:
        gabp.svm_create(p.X, p.y, p.gamma, p.C)
    assert ei.value.status == gabp.ENOMEM and "GB of device memory" in ei.value.message
    assert abs(_free_bytes() - free0) < (64 << 20)


def test_injected_alloc_failure(monkeypatch):
    """GABP_FAULT=alloc: create and the batch solve return GABP_ENOMEM with
    nothing left allocated; the server completes the request with
    GABP_ENOMEM and keeps serving; without the fault everything runs."""
    p = workloads.mixture(300, 6, seed=7)
    free0 = _free_bytes()
    monkeypatch.setenv("GABP_FAULT", "alloc")
    with pytest.raises(gabp.GabpError) as ei:
        gabp.svm_create(p.X, p.y, p.gamma, p.C)
    assert ei.value.status == gabp.ENOMEM and "injected" in ei.value.message
    with pytest.raises(gabp.GabpError) as ei:
        gabp.batch_solve([p, p], 10, 0.0)
    assert ei.value.status == gabp.ENOMEM
    srv = gabp.Server(iters=50, tol=1e-6, max_members=4)
    t = srv.submit(p.X, p.y, p.gamma, p.C)
    for _ in range(20):
        srv.step()
        if t in srv.completed():
            break
    _, r = srv.poll(t)
    assert r["status"] == gabp.ENOMEM
    monkeypatch.delenv("GABP_FAULT")
    t2 = srv.submit(p.X, p.y, p.gamma, p.C)
    res = None
    for _ in range(2000):
        srv.step()
        if t2 in srv.completed():
            res = srv.poll(t2)
            break
    srv.close()
    assert res is not None and res[1]["status"] == 0 and res[1]["converged"] == 1
    assert abs(_free_bytes() - free0) < (256 << 20)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    assert s.solve(10, 0.0)[2] == 10


def test_injected_nan_is_caught_by_the_staging_checks(monkeypatch):
    p = workloads.mixture(300, 6, seed=8)
    monkeypatch.setenv("GABP_FAULT", "nan")
    with pytest.raises(gabp.GabpError) as ei:
        gabp.svm_create(p.X, p.y, p.gamma, p.C)
    assert ei.value.status == gabp.EINVAL and "row 150" in ei.value.message


def test_injected_timeout_reaches_the_host_and_refit_recovers(monkeypatch):
    """GABP_FAULT=timeout: the solve reports GABP_ETIMEOUT (as when a bounded
    device wait runs out), the handle refuses further solves with
    GABP_ESTATE, and a refit restores it."""
    p = workloads.mixture(300, 6, seed=9)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    monkeypatch.setenv("GABP_FAULT", "timeout")
    with pytest.raises(gabp.GabpError) as ei:
        s.solve(20, 0.0)
    assert ei.value.status == gabp.ETIMEOUT
    monkeypatch.delenv("GABP_FAULT")
    with pytest.raises(gabp.GabpError) as ei:
        s.solve(20, 0.0)
    assert ei.value.status == gabp.ESTATE
    s.refit(p.X, p.y, p.gamma, p.C)
    alpha, rinf, k = s.solve(20, 0.0)
    assert k == 20 and np.all(np.isfinite(alpha))
