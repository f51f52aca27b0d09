"""gabp_decision_noalloc: decision values for callers that cannot allocate
device memory (plugins in host frameworks that own all device memory, loops
that cannot pay for cudaMalloc's synchronisation).

Checks, through the C ABI, that two calls in a row give the same values as
the handle-based gabp_svm_decision within the decision tolerance, and that
sizes beyond the fixed scratch maximum are refused with GABP_EINVAL.  This
file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu


def test_noalloc_decision_matches_handle_decision_twice():
    torch = pytest.importorskip("torch")
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()
    p = workloads.mixture(900, 24, seed=31, C=1.0)
    s = gabp.GabpSVM(p.X, p.y, p.gamma, p.C)
    alpha, _, _ = s.solve(20, 0.0)
    lam = s.stats()["lambda_"]
    Xd = torch.from_numpy(p.X).cuda()
    yd = torch.from_numpy(p.y).cuda()
    ad = torch.from_numpy(alpha).cuda()
    for call, seed in enumerate((32, 33)):
        Xt = workloads.test_points(p, 257 + call, seed=seed)
        ref = s.decision(Xt).astype(np.float64)
        out = torch.full((Xt.shape[0],), float("nan"), device="cuda")
        gabp.decision_noalloc(Xd, yd, ad, torch.from_numpy(Xt).cuda(), p.gamma, lam, out)
        got = out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), call
    s.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    torch = pytest.importorskip("torch")
    n, m, t = 20000, 4, 8000
    X = torch.zeros((n, m), device="cuda")
    y = torch.ones(n, device="cuda")
    a = torch.zeros(n, device="cuda")
    Xt = torch.zeros((t, m), device="cuda")
    out = torch.zeros(t, device="cuda")
    with pytest.raises(gabp.GabpError) as ei:
        gabp.decision_noalloc(X, y, a, Xt, 0.5, 0.0, out)
    assert ei.value.status == gabp.EINVAL and "scratch" in ei.value.message
