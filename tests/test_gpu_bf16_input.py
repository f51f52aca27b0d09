"""BF16 feature input (opts.x_dtype = 2): the rows are widened to FP32 on the
device, which is exact, so every result must equal bit for bit the one from
FP32 input holding the same values, in host and device pointer modes, for the
decision values, the precision form and the batched form; and the solve must
meet the FP32 bars against the FP64 oracle run on the BF16-rounded features
(Section 3's system for the data the caller holds)."""
import numpy as np
import pytest

import oracle
from paper_0810_1648_gb300 import gabp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL_MU = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_0810_1648_gb300 import build as gbuild
    gbuild.build()
    gabp.load()


def _bf16_case(n, m, seed):
    p = workloads.mixture(n, m, seed=seed, C=1.0)
    Xb = torch.from_numpy(p.X).to(torch.bfloat16)            # the caller's BF16 rows
    Xr = Xb.to(torch.float32).numpy()                        # the same values in FP32
    return p, Xb, Xr


@pytest.mark.parametrize("n,m", [(300, 9), (517, 33)])
def test_bf16_rows_equal_fp32_rows_of_the_same_values(n, m):
    p, Xb, Xr = _bf16_case(n, m, seed=41)
    ref = gabp.GabpSVM(Xr, p.y, p.gamma, p.C)
    a_ref, r_ref, k_ref = ref.solve(40, 0.0)
    host = gabp.GabpSVM(Xb, p.y, p.gamma, p.C)                          # host pointers
    a_h, r_h, k_h = host.solve(40, 0.0)
    dev = gabp.GabpSVM(Xb.cuda(), torch.from_numpy(p.y).cuda(), p.gamma, p.C)   # device pointers
    a_d, r_d, k_d = dev.solve(40, 0.0)
    assert host.x_dtype == 2 and dev.x_dtype == 2
    np.testing.assert_array_equal(a_ref, a_h)
    np.testing.assert_array_equal(a_ref, a_d.cpu().numpy())
    assert r_ref == r_h == r_d and k_ref == k_h == k_d
    # decision values from BF16 test rows, both modes
    Xt = workloads.test_points(p, 70, seed=42)
    Xtb = torch.from_numpy(Xt).to(torch.bfloat16)
    f_ref = ref.decision(Xtb.to(torch.float32).numpy())
    np.testing.assert_array_equal(f_ref, host.decision(Xtb))
    np.testing.assert_array_equal(f_ref, dev.decision(Xtb.cuda()).cpu().numpy())
    # a layout other than the handle's is refused by the binding
    with pytest.raises(TypeError):
        host.decision(Xt)


def test_bf16_rows_against_oracle():
    p, Xb, Xr = _bf16_case(700, 24, seed=43)
    s = gabp.GabpSVM(Xb.cuda(), torch.from_numpy(p.y).cuda(), p.gamma, p.C)
    s.solve(60, 0.0)
    mu = s.mean().cpu().numpy().astype(np.float64)
    X64 = Xr.astype(np.float64)
    Q = oracle.build_q(X64, p.y.astype(np.float64), p.gamma, p.C)
    r = oracle.gabp(Q, np.ones(p.n), iters=60, tol=0.0)
    assert np.max(np.abs(mu - r.mu)) / np.max(np.abs(r.mu)) <= REL_MU


def test_bf16_rows_precision_form_and_refit():
    p, Xb, Xr = _bf16_case(640, 64, seed=44)
    kw = dict(q_mode=gabp.Q_BF16, refine=10, msg_bf16=1)
    a_ref, _, _ = gabp.GabpSVM(Xr, p.y, p.gamma, p.C, **kw).solve(200, 1e-6)
    s = gabp.GabpSVM(Xb, p.y, p.gamma, p.C, **kw)
    a1, r1, _ = s.solve(200, 1e-6)
    np.testing.assert_array_equal(a_ref, a1)
    assert r1 < 1e-6
    q, Qb, Qr = _bf16_case(640, 64, seed=45)
    s.refit(Qb, q.y, q.gamma, q.C)
    a2, _, _ = s.solve(200, 1e-6)
    a2_ref, _, _ = gabp.GabpSVM(Qr, q.y, q.gamma, q.C, **kw).solve(200, 1e-6)
    np.testing.assert_array_equal(a2_ref, a2)


def test_bf16_rows_batched_form():
    cases = [_bf16_case(n, 16, seed=50 + k) for k, n in enumerate((150, 400, 999))]

    class Pb:
        def __init__(self, p, X):
            self.X, self.y, self.gamma, self.C = X, torch.from_numpy(p.y).cuda(), p.gamma, p.C

    a32, res32, rc32 = gabp.batch_solve([Pb(p, torch.from_numpy(Xr).cuda()) for p, _, Xr in cases], 30, 0.0, chunk=8)
    a16, res16, rc16 = gabp.batch_solve([Pb(p, Xb.cuda()) for p, Xb, _ in cases], 30, 0.0, chunk=8)
    assert rc32 == rc16 == gabp.OK
    for x, y_, r1, r2 in zip(a32, a16, res32, res16):
        np.testing.assert_array_equal(x.cpu().numpy(), y_.cpu().numpy())
        assert r1["residual_inf"] == r2["residual_inf"]
