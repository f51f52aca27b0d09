"""CPU-side checks of the C ABI: the library builds, loads and exports every
function the header declares; argument checks fail before any device work;
without a GPU every call that needs one fails loudly (no CPU fallback)."""
import ctypes

import numpy as np
import pytest

from paper_0810_1648_gb300 import build as gbuild
from paper_0810_1648_gb300 import gabp


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gabp.load()


def test_exports_every_declared_symbol(lib):
    names = gabp.declared_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm
    assert lib.gabp_version() == 3


def test_opts_default(lib):
    o = gabp.opts_default()
    assert o.q_mode == gabp.Q_F32 and o.diag_rule == gabp.DIAG_DOMINANT
    assert o.diag_delta == pytest.approx(0.1) and o.chunk == 16 and o.ptr_mode == 0


def test_argument_errors_before_device_work(lib):
    X = np.zeros((4, 3), np.float32)
    y = np.array([1, -1, 1, -1], np.float32)
    h = ctypes.c_void_p()
    V = ctypes.c_void_p
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, 1.0, None) == gabp.EINVAL
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 1, 3, 1.0, 1.0, ctypes.byref(h)) == gabp.EINVAL
    assert b"n >= 2" in lib.gabp_last_error()
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, -1.0, 1.0, ctypes.byref(h)) == gabp.EINVAL
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, 0.0, ctypes.byref(h)) == gabp.EINVAL
    assert lib.gabp_svm_create(None, V(y.ctypes.data), 4, 3, 1.0, 1.0, ctypes.byref(h)) == gabp.EINVAL
    o = gabp.opts_default(q_mode=7)
    assert lib.gabp_svm_create_ex(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, 1.0,
                                  ctypes.byref(o), ctypes.byref(h)) == gabp.EINVAL
    # gamma and lambda^2 enter the kernels in FP32: values beyond its range are refused
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1e39, 1.0, ctypes.byref(h)) == gabp.EINVAL
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, float("inf"),
                               ctypes.byref(h)) == gabp.EINVAL
    for bad in (dict(task=2), dict(stages=17), dict(stages=-1), dict(msg_bf16=1), dict(refine=65),
                dict(bias_mode=1, bias_lambda=2e19), dict(bias_mode=1, bias_lambda=-1.0),
                dict(x_dtype=3), dict(x_dtype=-1), dict(ptr_mode=2)):
        o = gabp.opts_default(**bad)
        assert lib.gabp_svm_create_ex(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, 1.0,
                                      ctypes.byref(o), ctypes.byref(h)) == gabp.EINVAL, bad
    cfg = gabp.ServerCfg()
    cfg.max_members = 4
    cfg.opts = gabp.opts_default(stages=99)
    srv = ctypes.c_void_p()
    assert lib.gabp_server_create(ctypes.byref(cfg), ctypes.byref(srv)) == gabp.EINVAL
    # null handles and outputs
    assert lib.gabp_svm_solve(None, 1, 0.0, None, None, None) == gabp.EINVAL
    assert lib.gabp_svm_destroy(None) == gabp.OK
    assert lib.gabp_server_completed(None, None, 0, None) == gabp.EINVAL
    assert lib.gabp_server_phases(None, None) == gabp.EINVAL


def test_no_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X = np.random.default_rng(0).standard_normal((8, 3)).astype(np.float32)
    y = np.array([1, -1] * 4, np.float32)
    with pytest.raises(gabp.GabpError) as ei:
        gabp.svm_create(X, y, 0.5, 1.0)
    assert ei.value.status == gabp.ECUDA


def test_noalloc_binding_rejects_bad_arguments():
    """decision_noalloc checks dtype, device and shapes before the call: a CPU
    or float64 tensor, or mismatched sizes, never reach the kernels."""
    torch = pytest.importorskip("torch")
    X = torch.zeros((8, 3))
    y, a = torch.ones(8), torch.zeros(8)
    Xt, out = torch.zeros((5, 3)), torch.zeros(5)
    with pytest.raises(gabp.GabpError) as ei:
        gabp.decision_noalloc(X, y, a, Xt, 0.5, 0.0, out)
    assert ei.value.status == gabp.EINVAL and "CUDA" in ei.value.message
    with pytest.raises(gabp.GabpError) as ei:
        gabp.decision_noalloc(np.zeros((8, 3), np.float32), y, a, Xt, 0.5, 0.0, out)
    assert ei.value.status == gabp.EINVAL


def test_unknown_fault_token_rejected_before_device_work(lib, monkeypatch):
    """GABP_FAULT (host-side fault injection) is parsed before any device
    call: an unknown token is GABP_EINVAL, with or without a GPU."""
    X = np.zeros((4, 3), np.float32)
    y = np.array([1, -1, 1, -1], np.float32)
    h = ctypes.c_void_p()
    V = ctypes.c_void_p
    monkeypatch.setenv("GABP_FAULT", "alloc,bogus")
    assert lib.gabp_svm_create(V(X.ctypes.data), V(y.ctypes.data), 4, 3, 1.0, 1.0, ctypes.byref(h)) == gabp.EINVAL
    assert b"GABP_FAULT" in lib.gabp_last_error()
    pr = (gabp.Problem * 1)(gabp.Problem(X.ctypes.data, y.ctypes.data, 4, 3, 1.0, 1.0))
    res = (gabp.Result * 1)()
    assert lib.gabp_batch_solve(pr, 1, None, 5, 0.0, res) == gabp.EINVAL
    assert b"GABP_FAULT" in lib.gabp_last_error()


def test_known_fault_tokens_do_not_mask_a_missing_device(lib, monkeypatch):
    """With a valid GABP_FAULT and no GPU, create still fails loudly with
    GABP_ECUDA (the injection sits behind the device checks)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X = np.random.default_rng(0).standard_normal((8, 3)).astype(np.float32)
    y = np.array([1, -1] * 4, np.float32)
    for tok in ("alloc", "nan", "timeout", "alloc,nan"):
        monkeypatch.setenv("GABP_FAULT", tok)
        with pytest.raises(gabp.GabpError) as ei:
            gabp.svm_create(X, y, 0.5, 1.0)
        assert ei.value.status == gabp.ECUDA, tok


def test_binding_input_layouts():
    """The binding maps torch dtypes onto opts.x_dtype and keeps later rows in
    the layout the handle was created with (no handle needed: the check is
    host-side marshalling)."""
    torch = pytest.importorskip("torch")
    assert gabp._torch_x_dtype(torch.zeros(2, 2)) == 0
    assert gabp._torch_x_dtype(torch.zeros(2, 2, dtype=torch.float64)) == 1
    assert gabp._torch_x_dtype(torch.zeros(2, 2, dtype=torch.bfloat16)) == 2
    with pytest.raises(TypeError):
        gabp._torch_x_dtype(torch.zeros(2, 2, dtype=torch.float16))
    s = object.__new__(gabp.GabpSVM)
    s.h = None
    s.x_dtype = 1
    x = s._x(np.ones((3, 2), np.float32))          # numpy rows are converted to the handle's layout
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
    with pytest.raises(TypeError):
        s._x(torch.ones(3, 2))                      # torch rows must already have it
    s.x_dtype = 2
    with pytest.raises(TypeError):
        s._x(np.ones((3, 2), np.float32))           # numpy has no BF16: such handles take torch rows
    t = torch.ones(3, 2, dtype=torch.bfloat16)
    assert s._x(t) is t
