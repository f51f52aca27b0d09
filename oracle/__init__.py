"""FP64 CPU oracle for the GaBP SVM solver (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never imports or
loads it, and it shares no code with ``paper_0810_1648_gb300``.

The arithmetic lives in ``gabp_oracle.c`` (plain C, FP64); this module builds it
with gcc on first use (``build()``) and wraps each function with ctypes and
numpy arrays.  See the C file for the paper passage behind every function.

Parity pins: every function here is checked by ``tests/test_oracle_pins.py``
against closed forms, library routines (numpy/scipy) or invariants, except the
two readings noted in the C file header that the paper leaves open (the amount
``delta`` of diagonal weighting and the support-vector threshold): those two
constants are "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DIAG_DOMINANT = 0
DIAG_SOFT2 = 1


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile gabp_oracle.c into liboracle.so (gcc, OpenMP, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    L, i32, f64 = ctypes.c_long, ctypes.c_int, ctypes.c_double
    sig = {
        "orc_threads": (i32, []),
        "orc_set_threads": (None, [i32]),
        "orc_q_offdiag": (f64, [D, D, f64, f64, L, f64, f64]),
        "orc_q_diag": (f64, [f64, f64, f64, i32, f64]),
        "orc_build_q": (i32, [D, D, L, L, f64, f64, f64, i32, f64, D]),
        "orc_gabp_info": (i32, [D, D, L, i32, f64, D, D, I, D, D, D, D]),
        "orc_gabp_literal": (i32, [D, D, L, i32, D, D]),
        "orc_gabp_staged": (i32, [D, D, L, i32, f64, i32, L, D, D, I, D, D, D, D]),
        "orc_stage_bounds": (None, [L, i32, ctypes.POINTER(ctypes.c_long)]),
        "orc_gabp_alg1": (i32, [D, D, L, i32, D, D]),
        "orc_pair_update": (None, [f64, f64, f64, f64, f64, D, D]),
        "orc_cholesky_solve": (i32, [D, D, L, D]),
        "orc_q_row": (None, [D, D, L, L, f64, f64, f64, i32, f64, L, D]),
        "orc_q_diag_all": (i32, [D, D, L, L, f64, f64, f64, i32, f64, D, D]),
        "orc_q_diag_tilemax": (i32, [D, D, L, L, f64, f64, f64, i32, f64, L, D, D, D]),
        "orc_residual_tile_sparse": (f64, [D, D, L, L, f64, f64, D, L, ctypes.c_void_p, D, D]),
        "orc_rows_tile_sparse": (i32, [D, D, L, L, f64, f64, f64, i32, f64, L, f64, ctypes.POINTER(ctypes.c_long), L,
                                       D, D, D, D, D]),
        "orc_cg_rbf": (i32, [D, D, L, L, f64, f64, f64, i32, f64, D, f64, i32, D, I]),
        "orc_dual_objective": (f64, [D, D, L]),
        "orc_decision": (i32, [D, D, D, L, L, D, L, f64, f64, D]),
        "orc_boxqp_bruteforce": (i32, [D, L, f64, f64, D, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _d(a):
    """Contiguous float64 copy/view of `a` and its ctypes pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc == 1:
        raise OracleError(f"{what}: nonpositive or non-finite cavity precision")
    if rc == 2:
        raise OracleError(f"{what}: out of memory")
    if rc == 3:
        raise OracleError(f"{what}: invalid argument")


def threads() -> int:
    return int(_load().orc_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def default_lambda(n: int) -> float:
    """Bias feature value 1/N (Section 3)."""
    return 1.0 / n


def build_q(X, y, gamma, C, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    """Dense FP64 Q (n x n) of the SVM dual with the weighted diagonal."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    Q = np.empty((n, n))
    rc = _load().orc_build_q(px, py, n, m, gamma, lam, C, diag_rule, delta,
                             Q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "build_q")
    return Q


def q_offdiag(xi, xj, yi, yj, gamma, lam):
    xi, pi = _d(xi)
    xj, pj = _d(xj)
    return float(_load().orc_q_offdiag(pi, pj, yi, yj, xi.shape[0], gamma, lam))


def q_diag(row_abs_sum, lam, C, diag_rule=DIAG_DOMINANT, delta=0.1):
    return float(_load().orc_q_diag(row_abs_sum, lam, C, diag_rule, delta))


def q_row(X, y, i, gamma, C, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    row = np.empty(n)
    _load().orc_q_row(px, py, n, m, gamma, lam, C, diag_rule, delta, int(i),
                      row.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return row


def q_diag_all(X, y, gamma, C, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    """(diag, R): Q_ii and R_i = sum_{j != i} |Q_ij| of every row, Q not stored."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    diag, R = np.empty(n), np.empty(n)
    rc = _load().orc_q_diag_all(px, py, n, m, gamma, lam, C, diag_rule, delta,
                                diag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "q_diag_all")
    return diag, R


def q_diag_tilemax(X, y, gamma, C, block=128, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    """(diag, R, tmax): as q_diag_all, plus the largest |Q_ij| of every
    block x block tile of the upper triangle (pairs i < j), as an Nt x Nt
    array with tmax[I, J] for I <= J (0 below the diagonal), Q not stored."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    nt = (n + block - 1) // block
    diag, R, flat = np.empty(n), np.empty(n), np.empty(nt * (nt + 1) // 2)
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_q_diag_tilemax(px, py, n, m, gamma, lam, C, diag_rule, delta, int(block),
                                    diag.ctypes.data_as(P), R.ctypes.data_as(P), flat.ctypes.data_as(P))
    _check(rc, "q_diag_tilemax")
    tmax = np.zeros((nt, nt))
    iu = np.triu_indices(nt)
    tmax[iu] = flat          # row-major upper triangle: L = I Nt - I (I - 1) / 2 + (J - I)
    return diag, R, tmax


def residual_tile_sparse(X, y, gamma, diag, keep, mu, block=128, lam=None):
    """r = 1 - Q mu (FP64) for the tile-sparse matrix with diagonal `diag` and
    the kept tiles keep[I, J] (I <= J, upper triangle), visiting kept tiles
    only.  Returns (r, ||r||_inf)."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    diag, pd = _d(diag)
    mu, pm = _d(mu)
    kp = np.ascontiguousarray(np.triu(np.asarray(keep, dtype=bool)), dtype=np.uint8)
    r = np.empty(n)
    rinf = _load().orc_residual_tile_sparse(px, py, n, m, gamma, lam, pd, int(block), kp.ctypes.data, pm,
                                            r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return r, float(rinf)


def rows_tile_sparse(X, y, gamma, C, tau, rows, mu, block=128, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    """For the chosen rows only (matrices too large for the whole-matrix
    passes): (tmax, R, diag, r) with tmax[k, J] the largest |Q| of tile (I, J)
    of row k's block row I, R[k] = sum_{j != i} |Q_ij| over the whole row,
    diag[k] the diagonal rule's Q_ii, and r[k] = 1 - (Q mu)_i of the tile-sparse
    matrix (tiles (I, J) with J == I or tmax > tau), all in FP64."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    mu, pm = _d(mu)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nt = (n + block - 1) // block
    k = rows.shape[0]
    tmax, R, diag, r = np.empty((k, nt)), np.empty(k), np.empty(k), np.empty(k)
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_rows_tile_sparse(px, py, n, m, gamma, lam, C, diag_rule, delta, int(block), float(tau),
                                      rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), k, pm,
                                      tmax.ctypes.data_as(P), R.ctypes.data_as(P), diag.ctypes.data_as(P),
                                      r.ctypes.data_as(P))
    _check(rc, "rows_tile_sparse")
    return tmax, R, diag, r


class GabpResult:
    def __init__(self, mu, Pt, kstar, rinf, rhist, Pin=None, Hin=None):
        self.mu, self.Pt, self.kstar, self.rinf, self.rhist = mu, Pt, kstar, rinf, rhist
        self.Pin, self.Hin = Pin, Hin   # Pin[i, k] = P_ki, Hin[i, k] = H_ki

    def alpha(self, C):
        """Output clip of the means to the box [0, C]."""
        return np.clip(self.mu, 0.0, C)


def gabp(Q, b=None, iters=100, tol=0.0, keep_messages=False):
    """Algorithm 2, synchronous, information form (see gabp_oracle.c)."""
    Q, pq = _d(Q)
    n = Q.shape[0]
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    mu, Pt = np.empty(n), np.empty(n)
    rhist = np.full(iters + 1, np.nan)
    k = ctypes.c_int(0)
    rinf = ctypes.c_double(0)
    Pin = np.empty((n, n)) if keep_messages else None
    Hin = np.empty((n, n)) if keep_messages else None
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_gabp_info(
        pq, pb, n, int(iters), float(tol), mu.ctypes.data_as(P), Pt.ctypes.data_as(P),
        ctypes.byref(k), ctypes.byref(rinf), rhist.ctypes.data_as(P),
        Pin.ctypes.data_as(P) if keep_messages else None,
        Hin.ctypes.data_as(P) if keep_messages else None)
    _check(rc, "gabp")
    return GabpResult(mu, Pt, k.value, rinf.value, rhist[: k.value + 1], Pin, Hin)


def gabp_literal(Q, b=None, iters=10):
    """Algorithm 2 with the message means as state (divides by Q_ij)."""
    Q, pq = _d(Q)
    n = Q.shape[0]
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    mu, Pt = np.empty(n), np.empty(n)
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_gabp_literal(pq, pb, n, int(iters), mu.ctypes.data_as(P),
                                  Pt.ctypes.data_as(P))
    _check(rc, "gabp_literal")
    return mu, Pt


def gabp_alg1(Q, b=None, iters=10):
    """Algorithm 1 (pairwise GaBP with explicit exclusion sums)."""
    Q, pq = _d(Q)
    n = Q.shape[0]
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    mu, Pt = np.empty(n), np.empty(n)
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_gabp_alg1(pq, pb, n, int(iters), mu.ctypes.data_as(P),
                               Pt.ctypes.data_as(P))
    _check(rc, "gabp_alg1")
    return mu, Pt


def pair_update(q, Pt_i, ht_i, Pt_j, ht_j, msg):
    """New (P_ij, P_ji, H_ij, H_ji) of one pair from its old state."""
    msg, pm = _d(msg)
    out = np.empty(4)
    _load().orc_pair_update(float(q), float(Pt_i), float(ht_i), float(Pt_j),
                            float(ht_j), pm,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def cholesky_solve(Q, b=None):
    Q, pq = _d(Q)
    n = Q.shape[0]
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    x = np.empty(n)
    rc = _load().orc_cholesky_solve(pq, pb, n, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(rc, "cholesky_solve")
    return x


def cg_rbf(X, y, gamma, C, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1, b=None,
           rtol=1e-12, maxit=500):
    """Matrix-free FP64 CG for Q alpha = b with Q formed row by row."""
    X, px = _d(X)
    y, py = _d(y)
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    x = np.empty(n)
    its = ctypes.c_int(0)
    rc = _load().orc_cg_rbf(px, py, n, m, gamma, lam, C, diag_rule, delta, pb, rtol,
                            maxit, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            ctypes.byref(its))
    _check(rc, "cg_rbf")
    return x, its.value


def dual_objective(Q, h):
    Q, pq = _d(Q)
    h, ph = _d(h)
    return float(_load().orc_dual_objective(pq, ph, Q.shape[0]))


def decision(X, y, h, Xt, gamma, lam=None):
    """f(x) = sum_i h_i y_i (K(x_i, x) + lambda^2) for every row of Xt."""
    X, px = _d(X)
    y, py = _d(y)
    h, ph = _d(h)
    Xt, pt = _d(np.atleast_2d(Xt))
    n, m = X.shape
    lam = default_lambda(n) if lam is None else lam
    f = np.empty(Xt.shape[0])
    _load().orc_decision(px, py, ph, n, m, pt, Xt.shape[0], gamma, lam,
                         f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return f


def boxqp_bruteforce(Q, C, kkt_tol=1e-10):
    """Exact minimiser of 1/2 a'Qa - 1'a on [0, C]^n, n <= 12."""
    Q, pq = _d(Q)
    n = Q.shape[0]
    a = np.empty(n)
    nk = ctypes.c_int(0)
    rc = _load().orc_boxqp_bruteforce(pq, n, float(C), float(kkt_tol),
                                      a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(nk))
    _check(rc, "boxqp_bruteforce")
    return a, nk.value


def solve_svm(X, y, gamma, C, iters=200, tol=1e-6, lam=None,
              diag_rule=DIAG_DOMINANT, delta=0.1):
    """Whole solve as the paper runs it: Q, then Algorithm 2 with b = 1.

    Returns (Q, GabpResult); alpha = result.alpha(C), support vectors are the
    indices with alpha > 0 (threshold 0 on the clipped weights).
    """
    Q = build_q(X, y, gamma, C, lam, diag_rule, delta)
    return Q, gabp(Q, np.ones(Q.shape[0]), iters, tol)


def build_q_krr(X, gamma, ridge, lam=0.0, diag_rule=DIAG_DOMINANT, delta=0.1):
    """Dense FP64 matrix of kernel ridge regression (Section 1.2) on the same
    kernel: off-diagonal K_ij (+ lam^2 with the bias feature on), diagonal
    K_ii + ridge = 1 + ridge under the soft2 rule, raised to (1 + delta) times
    the row's off-diagonal sum under the dominant rule (Section 3.1 weighting).
    No labels enter the matrix; the ridge takes the place of 1/C."""
    X = np.asarray(X, dtype=np.float64)
    return build_q(X, np.ones(X.shape[0]), gamma, 1.0 / ridge, lam, diag_rule, delta)


def solve_krr(X, t, gamma, ridge, iters=200, tol=1e-6, lam=0.0,
              diag_rule=DIAG_DOMINANT, delta=0.1):
    """KRR solve: the matrix above, then Algorithm 2 with b = the targets.
    Returns (Q, GabpResult); the coefficients are result.mu (unclipped) and
    the prediction is f(x) = sum_i c_i (K(x_i, x) + lam^2)."""
    Q = build_q_krr(X, gamma, ridge, lam, diag_rule, delta)
    return Q, gabp(Q, np.asarray(t, dtype=np.float64), iters, tol)


def stage_bounds(nt: int, stages: int):
    """Block boundaries B[0..S] of the staged schedule (see gabp_oracle.c)."""
    B = (ctypes.c_long * (stages + 1))()
    _load().orc_stage_bounds(int(nt), int(stages), B)
    return list(B)


def gabp_staged(Q, b=None, iters=100, tol=0.0, stages=2, block=128, keep_messages=False):
    """Algorithm 2 under the block Gauss-Seidel schedule (stages = 1: synchronous)."""
    Q, pq = _d(Q)
    n = Q.shape[0]
    b = np.ones(n) if b is None else b
    b, pb = _d(b)
    mu, Pt = np.empty(n), np.empty(n)
    rhist = np.full(iters + 1, np.nan)
    k = ctypes.c_int(0)
    rinf = ctypes.c_double(0)
    Pin = np.empty((n, n)) if keep_messages else None
    Hin = np.empty((n, n)) if keep_messages else None
    P = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_gabp_staged(
        pq, pb, n, int(iters), float(tol), int(stages), int(block), mu.ctypes.data_as(P), Pt.ctypes.data_as(P),
        ctypes.byref(k), ctypes.byref(rinf), rhist.ctypes.data_as(P),
        Pin.ctypes.data_as(P) if keep_messages else None, Hin.ctypes.data_as(P) if keep_messages else None)
    _check(rc, "gabp_staged")
    return GabpResult(mu, Pt, k.value, rinf.value, rhist[:k.value + 1], Pin, Hin)


def build_q_tile_sparse(X, y, gamma, C, tau, block=128, lam=None, diag_rule=DIAG_DOMINANT, delta=0.1):
    """The SVM matrix with the tile-sparse reading of Section 6's sparsified
    kernel: the off-diagonal entries are grouped in block x block tiles of the
    upper triangle (and their mirrors); a tile whose largest |Q_ij| is <= tau
    is dropped (all its entries 0), diagonal tiles are always kept, and the
    diagonal keeps its value from the whole matrix (the rule on all row sums),
    so only the dropped entries change.  Returns (Q, keep) with keep[I, J] for
    I <= J."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    lam_v = default_lambda(n) if lam is None else lam
    Q = build_q(X, y, gamma, C, lam_v, diag_rule, delta)
    nt = (n + block - 1) // block
    keep = np.zeros((nt, nt), dtype=bool)
    for I in range(nt):
        for J in range(I, nt):
            sl_i, sl_j = slice(I * block, (I + 1) * block), slice(J * block, (J + 1) * block)
            B = np.abs(Q[sl_i, sl_j])
            if I == J:
                B = np.triu(B, 1)
            keep[I, J] = I == J or B.max() > tau
            if not keep[I, J]:
                Q[sl_i, sl_j] = 0.0
                Q[sl_j, sl_i] = 0.0
    return Q, keep
