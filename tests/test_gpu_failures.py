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
