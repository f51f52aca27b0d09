"""Python binding of libgabp_svm.so (the C ABI in include/gabp_svm.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Host inputs are numpy arrays (copied by the library); device
inputs are torch CUDA tensors (``ptr_mode=1``), for which torch supplies the
memory and the library reads it in place.  There is no CPU fallback: without
the built library or a GPU every call raises.

Function names follow the C ABI (``svm_create`` wraps ``gabp_svm_create_ex``
and so on); ``GabpSVM`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgabp_svm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gabp_svm.h")

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, ESTATE = range(7)
STATUS_NAMES = {0: "GABP_OK", 1: "GABP_EINVAL", 2: "GABP_ENOMEM", 3: "GABP_ECUDA",
                4: "GABP_ENUMERIC", 5: "GABP_ETIMEOUT", 6: "GABP_ESTATE"}
Q_F32, Q_BF16, Q_RECOMPUTE = 0, 1, 2
DIAG_DOMINANT, DIAG_SOFT2 = 0, 1
TASK_SVM, TASK_KRR = 0, 1


class GabpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Opts(ctypes.Structure):
    _fields_ = [("x_dtype", ctypes.c_int32), ("ptr_mode", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("diag_rule", ctypes.c_int32),
                ("diag_delta", ctypes.c_double), ("bias_mode", ctypes.c_int32),
                ("bias_lambda", ctypes.c_double), ("q_mode", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("sv_threshold", ctypes.c_double),
                ("chunk", ctypes.c_int32), ("msg_bf16", ctypes.c_int32),
                ("refine_handover", ctypes.c_float), ("refine_inner", ctypes.c_float),
                ("task", ctypes.c_int32), ("stages", ctypes.c_int32), ("sparse_tau", ctypes.c_float),
                ("reserved", ctypes.c_int32 * 1)]


class Profile(ctypes.Structure):
    _fields_ = [("sweep_launches", ctypes.c_int64), ("sweep_launches_zero_state", ctypes.c_int64),
                ("sweep_launches_p_frozen", ctypes.c_int64),
                ("sweep_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("sweeps_total", ctypes.c_int64),
                ("kstar", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("residual_inf", ctypes.c_double), ("dual_objective", ctypes.c_double),
                ("n_support", ctypes.c_int64), ("lambda_", ctypes.c_double),
                ("gamma", ctypes.c_double), ("C", ctypes.c_double), ("diag_delta", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("q_mode", ctypes.c_int32),
                ("diag_rule", ctypes.c_int32), ("refine_passes", ctypes.c_int32),
                ("tiles_total", ctypes.c_int64), ("tiles_kept", ctypes.c_int64),
                ("margin", ctypes.c_double), ("err_bound", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("m", ctypes.c_int64), ("gamma", ctypes.c_double), ("C", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_void_p), ("residual_inf", ctypes.c_double),
                ("dual_objective", ctypes.c_double), ("n_support", ctypes.c_int64),
                ("iters_done", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("refine_passes", ctypes.c_int32),
                ("mu", ctypes.c_void_p), ("margin", ctypes.c_double), ("err_bound", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("alpha", "mu")}


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_members", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("tol", ctypes.c_double), ("opts", Opts)]


_lib = None


def declared_functions() -> list[str]:
    """Names of every function include/gabp_svm.h exports."""
    text = open(HEADER).read()
    return re.findall(r"GABP_API\s+[\w\s\*]+?\b(gabp_\w+)\s*\(", text)


def load():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0810_1648_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    V, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER
    st = ctypes.c_int
    sigs = {
        "gabp_svm_opts_default": (None, [P(Opts)]),
        "gabp_svm_create": (st, [V, V, I64, I64, D, D, P(V)]),
        "gabp_svm_create_ex": (st, [V, V, I64, I64, D, D, P(Opts), P(V)]),
        "gabp_svm_refit": (st, [V, V, V, D, D]),
        "gabp_svm_solve": (st, [V, I32, D, V, P(D), P(I32)]),
        "gabp_svm_get_mean": (st, [V, V]),
        "gabp_svm_decision": (st, [V, V, I64, V]),
        "gabp_svm_support": (st, [V, V, I64, P(I64)]),
        "gabp_svm_get_stats": (st, [V, P(Stats)]),
        "gabp_svm_get_q": (st, [V, V]),
        "gabp_svm_get_pairs": (st, [V, V, V, I64, V]),
        "gabp_svm_get_aggregates": (st, [V, V, V, V]),
        "gabp_svm_set_profiling": (st, [V, I32]),
        "gabp_svm_get_profile": (st, [V, P(Profile), I32]),
        "gabp_svm_destroy": (st, [V]),
        "gabp_decision_noalloc": (st, [V, V, V, I64, I64, V, I64, D, D, V, V]),
        "gabp_selftest_bounded_wait": (st, [I64]),
        "gabp_selftest_reciprocal": (st, [V, V, I64]),
        "gabp_batch_solve": (st, [P(Problem), I64, P(Opts), I32, D, P(Result)]),
        "gabp_batch_last_phases": (st, [V]),
        "gabp_batch_release": (st, []),
        "gabp_server_create": (st, [P(ServerCfg), P(V)]),
        "gabp_server_submit": (st, [V, P(Problem), V, P(I64)]),
        "gabp_server_submit_ex": (st, [V, P(Problem), V, V, P(I64)]),
        "gabp_server_step": (st, [V, P(I32), P(I32), P(I32)]),
        "gabp_server_poll": (st, [V, I64, P(Result), P(I32)]),
        "gabp_server_completed": (st, [V, V, I32, P(I32)]),
        "gabp_server_phases": (st, [V, V]),
        "gabp_server_destroy": (st, [V]),
        "gabp_last_error": (ctypes.c_char_p, []),
        "gabp_version": (I32, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        raise GabpError(rc, load().gabp_last_error().decode(errors="replace"))


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Raw address of a numpy array or torch tensor (which must be contiguous)."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _is_cuda(a) -> bool:
    return _is_torch(a) and a.is_cuda


def _sync_torch(*arrays):
    """Device inputs written on torch's stream must be complete before the
    library's stream reads them."""
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
            return


def opts_default(**kw) -> Opts:
    o = Opts()
    load().gabp_svm_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _torch_x_dtype(X) -> int:
    """opts.x_dtype of a torch feature tensor: 0 float32, 1 float64, 2 bfloat16."""
    import torch
    codes = {torch.float32: 0, torch.float64: 1, torch.bfloat16: 2}
    if X.dtype not in codes:
        raise TypeError("X must be float32, float64 or bfloat16")
    return codes[X.dtype]


def _prep_x(X, device_mode):
    if device_mode:
        return X.contiguous(), _torch_x_dtype(X)
    X = np.asarray(X)
    if X.dtype not in (np.float32, np.float64):
        X = X.astype(np.float32)
    return np.ascontiguousarray(X), (1 if X.dtype == np.float64 else 0)


def svm_create(X, y, gamma: float, C: float, opts: Opts | None = None):
    """gabp_svm_create_ex: returns an opaque handle (int).  X as a torch CUDA
    tensor selects device-pointer mode; numpy arrays or (pinned) torch CPU
    tensors select host-pointer mode."""
    device_mode = _is_cuda(X)
    if _is_torch(X) and not device_mode:
        import torch
        o = opts if opts is not None else opts_default()
        o.x_dtype = _torch_x_dtype(X)
        o.ptr_mode = 0
        y = torch.as_tensor(y, dtype=torch.float32).contiguous()
        h = ctypes.c_void_p()
        _check(load().gabp_svm_create_ex(_ptr(X.contiguous()), _ptr(y), X.shape[0], X.shape[1],
                                         float(gamma), float(C), ctypes.byref(o), ctypes.byref(h)))
        return h.value
    X, x_dtype = _prep_x(X, device_mode)
    o = opts if opts is not None else opts_default()
    o.x_dtype = x_dtype
    o.ptr_mode = 1 if device_mode else 0
    if device_mode:
        import torch
        y = y.to(device=X.device, dtype=torch.float32).contiguous()
        _sync_torch(X, y)
    else:
        y = np.ascontiguousarray(y, dtype=np.float32)
    h = ctypes.c_void_p()
    n, m = X.shape
    _check(load().gabp_svm_create_ex(_ptr(X), _ptr(y), n, m, float(gamma), float(C),
                                     ctypes.byref(o), ctypes.byref(h)))
    return h.value


def svm_refit(h, X, y, gamma: float, C: float):
    _sync_torch(X, y)
    _check(load().gabp_svm_refit(ctypes.c_void_p(h), _ptr(X), _ptr(y), float(gamma), float(C)))


def svm_solve(h, iters: int, tol: float, alpha_out):
    """gabp_svm_solve into alpha_out (numpy float32 or torch CUDA float32).
    Returns (residual_inf, iters_done)."""
    r = ctypes.c_double(0)
    k = ctypes.c_int32(0)
    _check(load().gabp_svm_solve(ctypes.c_void_p(h), int(iters), float(tol), _ptr(alpha_out),
                                 ctypes.byref(r), ctypes.byref(k)))
    return r.value, k.value


def svm_get_mean(h, out):
    _check(load().gabp_svm_get_mean(ctypes.c_void_p(h), _ptr(out)))


def svm_decision(h, Xt, out):
    _sync_torch(Xt)
    _check(load().gabp_svm_decision(ctypes.c_void_p(h), _ptr(Xt), int(Xt.shape[0]), _ptr(out)))


def svm_support(h, n: int) -> np.ndarray:
    idx = np.empty(n, dtype=np.int32)
    cnt = ctypes.c_int64(0)
    _check(load().gabp_svm_support(ctypes.c_void_p(h), _ptr(idx), n, ctypes.byref(cnt)))
    return idx[: cnt.value].copy()


def svm_get_stats(h) -> dict:
    s = Stats()
    _check(load().gabp_svm_get_stats(ctypes.c_void_p(h), ctypes.byref(s)))
    return s.as_dict()


def svm_get_q(h, n: int) -> np.ndarray:
    Q = np.empty((n, n), dtype=np.float32)
    _check(load().gabp_svm_get_q(ctypes.c_void_p(h), _ptr(Q)))
    return Q


def svm_get_pairs(h, i, j) -> np.ndarray:
    i = np.ascontiguousarray(i, dtype=np.int64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    out = np.empty((len(i), 4), dtype=np.float32)
    _check(load().gabp_svm_get_pairs(ctypes.c_void_p(h), _ptr(i), _ptr(j), len(i), _ptr(out)))
    return out


def svm_get_aggregates(h, n: int):
    Pt, ht, mu = (np.empty(n, dtype=np.float32) for _ in range(3))
    _check(load().gabp_svm_get_aggregates(ctypes.c_void_p(h), _ptr(Pt), _ptr(ht), _ptr(mu)))
    return Pt, ht, mu


def svm_set_profiling(h, on):
    """on: False / 0 off, True / 1 every round's pair sweep timed, k > 1 every k-th round's."""
    _check(load().gabp_svm_set_profiling(ctypes.c_void_p(h), int(on)))


def svm_get_profile(h, reset: bool = False) -> dict:
    p = Profile()
    _check(load().gabp_svm_get_profile(ctypes.c_void_p(h), ctypes.byref(p), 1 if reset else 0))
    return p.as_dict()


def _check_noalloc_args(X, y, alpha, Xt, out):
    """The arguments of decision_noalloc: contiguous float32 CUDA tensors on one
    device, X (n x m) and Xt (t x m) with the same m, y and alpha of length n,
    out of length t.  Raises GabpError(EINVAL) before any library call."""
    def bad(msg):
        raise GabpError(EINVAL, "decision_noalloc: " + msg)
    ts = {"X": X, "y": y, "alpha": alpha, "Xt": Xt, "out": out}
    for k, v in ts.items():
        if not _is_torch(v) or not v.is_cuda:
            bad(f"{k} must be a CUDA tensor")
        if str(v.dtype) != "torch.float32":
            bad(f"{k} must be float32 (got {v.dtype})")
        if not v.is_contiguous():
            bad(f"{k} must be contiguous")
    if len({v.device for v in ts.values()}) != 1:
        bad("all tensors must be on one device")
    if X.dim() != 2 or Xt.dim() != 2 or X.shape[1] != Xt.shape[1]:
        bad("X and Xt must be 2-D with the same number of columns")
    n, t = int(X.shape[0]), int(Xt.shape[0])
    if y.numel() != n or alpha.numel() != n:
        bad(f"y and alpha need {n} entries")
    if out.numel() != t:
        bad(f"out needs {t} entries")


def decision_noalloc(X, y, alpha, Xt, gamma: float, lam: float, out, stream=None):
    """gabp_decision_noalloc: torch CUDA float32 tensors, no allocation in the library."""
    _check_noalloc_args(X, y, alpha, Xt, out)
    _sync_torch(X, y, alpha, Xt)
    _check(load().gabp_decision_noalloc(_ptr(X), _ptr(y), _ptr(alpha), int(X.shape[0]), int(X.shape[1]),
                                        _ptr(Xt), int(Xt.shape[0]), float(gamma), float(lam), _ptr(out),
                                        ctypes.c_void_p(stream) if stream else None))


def selftest_bounded_wait(limit_ns: int) -> int:
    """Status of gabp_selftest_bounded_wait (GABP_ETIMEOUT when the wait works)."""
    rc = load().gabp_selftest_bounded_wait(int(limit_ns))
    return rc


def batch_solve(problems, iters: int, tol: float, means: bool = False, **opts):
    """gabp_batch_solve over a list of workloads.Problem-like objects: numpy X
    (float32/float64) and y, or torch CUDA tensors for all of them (X float32
    or bfloat16, one dtype for all; y float32; device pointer mode; alphas
    then come back as CUDA tensors).  Returns
    (list of alpha arrays, list of result dicts, overall status); with
    means=True each result dict also carries the unclipped means under "mu"
    (same array kind as alpha)."""
    probs = (Problem * len(problems))()
    keep, alphas, mus = [], [], []
    xcode = None   # opts.x_dtype shared by every problem
    dev = len(problems) > 0 and _is_cuda(problems[0].X)
    if dev:
        import torch
    for k, p in enumerate(problems):
        if dev:
            X = p.X.contiguous()
            y = p.y.contiguous()
            if y.dtype != torch.float32 or not y.is_cuda:
                raise TypeError("device-mode labels must be float32 CUDA tensors")
            xd = _torch_x_dtype(X)
            if xd == 1 or (xcode is not None and xcode != xd):
                raise TypeError("device-mode rows: one dtype (float32 or bfloat16) for all problems")
            xcode = xd
            keep += [X, y]
            probs[k] = Problem(X.data_ptr(), y.data_ptr(), X.shape[0], X.shape[1], float(p.gamma), float(p.C))
            alphas.append(torch.empty(X.shape[0], dtype=torch.float32, device=X.device))
            if means:
                mus.append(torch.empty(X.shape[0], dtype=torch.float32, device=X.device))
            continue
        X = np.ascontiguousarray(p.X)
        if xcode is None:
            xcode = 1 if X.dtype == np.float64 else 0
        X = X.astype(np.float64 if xcode == 1 else np.float32, copy=False)
        y = np.ascontiguousarray(p.y, dtype=np.float32)
        keep += [X, y]
        probs[k] = Problem(X.ctypes.data, y.ctypes.data, X.shape[0], X.shape[1], float(p.gamma), float(p.C))
        alphas.append(np.empty(X.shape[0], dtype=np.float32))
        if means:
            mus.append(np.empty(X.shape[0], dtype=np.float32))
    if dev:
        _sync_torch(*keep)
    res = (Result * len(problems))()
    for k in range(len(problems)):
        res[k].alpha = alphas[k].data_ptr() if dev else alphas[k].ctypes.data
        if means:
            res[k].mu = mus[k].data_ptr() if dev else mus[k].ctypes.data
    o = opts_default(**opts)
    o.x_dtype = xcode or 0
    if dev:
        o.ptr_mode = 1
    rc = load().gabp_batch_solve(probs, len(problems), ctypes.byref(o), int(iters), float(tol), res)
    if rc not in (OK, ENUMERIC):
        _check(rc)
    out = [res[k].as_dict() for k in range(len(problems))]
    if means:
        for d, mu in zip(out, mus):
            d["mu"] = mu
    return alphas, out, rc


def batch_release():
    """gabp_batch_release: frees this thread's kept batch engine."""
    _check(load().gabp_batch_release())


def batch_last_phases() -> dict:
    out = np.zeros(7)
    _check(load().gabp_batch_last_phases(_ptr(out)))
    return dict(zip(["form_ms", "tune_ms", "rounds_ms", "stop_ms", "total_ms", "chunks", "add_ms"], out.tolist()))


class Server:
    """Continuous-batching server (gabp_server_*), host-pointer mode."""

    def __init__(self, iters=200, tol=1e-6, budget_bytes=0, max_members=64, **opts):
        cfg = ServerCfg()
        cfg.hbm_budget_bytes = int(budget_bytes)
        cfg.max_members = int(max_members)
        cfg.iters = int(iters)
        cfg.tol = float(tol)
        cfg.opts = opts_default(**opts)
        self.h = ctypes.c_void_p()
        _check(load().gabp_server_create(ctypes.byref(cfg), ctypes.byref(self.h)))
        self._keep = {}

    def submit(self, X, y, gamma, C, means: bool = False):
        """Queues one problem; with means=True its poll() result dict also
        carries the unclipped means under "mu" (gabp_server_submit_ex)."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        alpha = np.empty(X.shape[0], dtype=np.float32)
        mu = np.empty(X.shape[0], dtype=np.float32) if means else None
        pr = Problem(X.ctypes.data, y.ctypes.data, X.shape[0], X.shape[1], float(gamma), float(C))
        t = ctypes.c_int64()
        _check(load().gabp_server_submit_ex(self.h, ctypes.byref(pr), ctypes.c_void_p(alpha.ctypes.data),
                                            ctypes.c_void_p(mu.ctypes.data) if means else None,
                                            ctypes.byref(t)))
        self._keep[t.value] = (X, y, alpha, mu)
        return t.value

    def step(self):
        a, q, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().gabp_server_step(self.h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(c)))
        return a.value, q.value, c.value

    def completed(self, cap=4096):
        """Tickets finished since the previous call."""
        buf = (ctypes.c_int64 * cap)()
        out = []
        while True:
            k = ctypes.c_int32()
            _check(load().gabp_server_completed(self.h, ctypes.cast(buf, ctypes.c_void_p), cap, ctypes.byref(k)))
            out.extend(buf[i] for i in range(k.value))
            if k.value < cap:
                return out

    def phases(self):
        """Host wall time (ms) per phase of the steps so far."""
        out = (ctypes.c_double * 8)()
        _check(load().gabp_server_phases(self.h, ctypes.cast(out, ctypes.c_void_p)))
        keys = ("admit_ms", "activate_ms", "rebuild_ms", "rounds_ms", "stop_ms", "total_ms", "steps", "rebuilds")
        return dict(zip(keys, list(out)))

    def poll(self, ticket):
        r = Result()
        d = ctypes.c_int32()
        _check(load().gabp_server_poll(self.h, int(ticket), ctypes.byref(r), ctypes.byref(d)))
        if not d.value:
            return None
        X, y, alpha, mu = self._keep.pop(ticket)
        d = r.as_dict()
        if mu is not None:
            d["mu"] = mu
        return alpha, d

    def close(self):
        if self.h:
            load().gabp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_reciprocal(d):
    """The sweep's reciprocal evaluated on the GPU for float32 inputs d."""
    d = np.ascontiguousarray(d, dtype=np.float32)
    out = np.empty_like(d)
    _check(load().gabp_selftest_reciprocal(_ptr(d), _ptr(out), d.size))
    return out


def svm_destroy(h):
    if h:
        _check(load().gabp_svm_destroy(ctypes.c_void_p(h)))


class GabpSVM:
    """Owning wrapper around one handle (host numpy inputs unless X is a torch
    CUDA tensor)."""

    def __init__(self, X, y, gamma: float, C: float, **opts):
        self.n, self.m = int(X.shape[0]), int(X.shape[1])
        self.device_mode = _is_cuda(X)
        self.C = float(C)
        o = opts_default(**opts)
        self.h = svm_create(X, y, gamma, C, o)
        self.x_dtype = int(o.x_dtype)   # the layout every later X / Xtest must have

    def _x(self, X):
        """X in the handle's layout (torch tensors are passed as they are and
        must already have it; numpy arrays are converted)."""
        if _is_torch(X):
            if _torch_x_dtype(X) != self.x_dtype:
                raise TypeError(f"X has {X.dtype}; this solver was created with x_dtype {self.x_dtype}")
            return X.contiguous()
        if self.x_dtype == 2:
            raise TypeError("this solver reads bfloat16 rows: pass a torch bfloat16 tensor")
        return np.ascontiguousarray(X, dtype=np.float64 if self.x_dtype == 1 else np.float32)

    def solve(self, iters: int = 200, tol: float = 1e-6):
        if self.device_mode:
            import torch
            alpha = torch.empty(self.n, dtype=torch.float32, device="cuda")
        else:
            alpha = np.empty(self.n, dtype=np.float32)
        rinf, k = svm_solve(self.h, iters, tol, alpha)
        return alpha, rinf, k

    def mean(self):
        out = np.empty(self.n, dtype=np.float32)
        if self.device_mode:
            import torch
            out = torch.empty(self.n, dtype=torch.float32, device="cuda")
        svm_get_mean(self.h, out)
        return out

    def decision(self, Xt):
        Xt = self._x(Xt)
        if self.device_mode:
            import torch
            out = torch.empty(Xt.shape[0], dtype=torch.float32, device="cuda")
        else:
            out = np.empty(Xt.shape[0], dtype=np.float32)
        svm_decision(self.h, Xt, out)
        return out

    def support(self):
        return svm_support(self.h, self.n)

    def stats(self):
        return svm_get_stats(self.h)

    def refit(self, X, y, gamma, C):
        self.C = float(C)
        X = self._x(X)
        if not _is_torch(y):
            y = np.ascontiguousarray(y, dtype=np.float32)
        svm_refit(self.h, X, y, gamma, C)

    def close(self):
        if self.h:
            svm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
