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
