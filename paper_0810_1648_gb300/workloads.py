"""Seeded synthetic SVM training sets shaped like the paper's workloads.

This module only draws random inputs (features X, labels y and the solver
parameters that go with them). It holds none of the GaBP arithmetic, so both
the CUDA path and the FP64 oracle may take their inputs from it.

Workloads (Section 5 of the paper runs RBF-kernel SVMs on UCI sets of up to
150,000 x 54 and 60,000 x 784; none of those data sets is available, so these
generators stand in for them):

* ``two_gaussians``   two classes, means +-shift*1, unit variance (the small
                      plain case, n=1000, m=10).
* ``mixture``         two classes, each a mixture of ``comps`` Gaussian
                      components whose means are drawn N(0, I) and whose
                      samples are mean + sigma*N(0, I) (n=20000, m=128; and
                      n=100000, m=64).
* ``batch_grid``      many uneven instances: n log-uniform in [200, 4000], m
                      from {8, 32, 128, 256}, a C x gamma grid per data set.
* ``poisson_requests`` arrival times and shapes of a stream of training
                      requests.
* ``clustered_mixture`` the mixture with rows grouped by component (the
                      input order the tile-sparse option needs).
* ``krr_targets``     real regression targets for the kernel ridge
                      regression task: a smooth random function of the
                      features plus noise.

Labels are +-1, rows are shuffled, every draw comes from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """One training set plus its RBF width and box constant (for the
    regression task: targets in y and the ridge in C)."""

    X: np.ndarray          # n x m, row-major
    y: np.ndarray          # n, float32: labels +-1 (SVM) or real targets (KRR)
    gamma: float           # RBF: K(a, b) = exp(-gamma * ||a - b||^2)
    C: float               # box constant 0 <= alpha <= C (SVM) or ridge lambda_r (KRR)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def m(self) -> int:
        return int(self.X.shape[1])


def _labels(n: int) -> np.ndarray:
    half = n // 2
    return np.concatenate([np.ones(n - half), -np.ones(half)]).astype(np.float32)


def two_gaussians(n: int = 1000, m: int = 10, seed: int = 0, shift: float = 0.5,
                  dtype=np.float64) -> Problem:
    """Class +1 ~ N(+shift*1, I), class -1 ~ N(-shift*1, I), rows shuffled."""
    rng = np.random.default_rng(seed)
    y = _labels(n)
    X = rng.standard_normal((n, m)) + shift * y[:, None].astype(np.float64)
    perm = rng.permutation(n)
    return Problem(X[perm].astype(dtype), y[perm].copy(), 1.0 / m, 1.0,
                   f"two_gaussians_n{n}_m{m}_s{seed}")


def mixture(n: int, m: int, seed: int, gamma: float | None = None, C: float = 1.0,
            comps: int = 3, sigma: float = 0.7, dtype=np.float32) -> Problem:
    """Two classes, each a mixture of `comps` components (means N(0, I))."""
    rng = np.random.default_rng(seed)
    y = _labels(n)
    means = rng.standard_normal((2, comps, m))
    cls = (y < 0).astype(np.int64)
    comp = rng.integers(0, comps, size=n)
    X = means[cls, comp] + sigma * rng.standard_normal((n, m))
    perm = rng.permutation(n)
    g = (1.0 / m) if gamma is None else gamma
    return Problem(X[perm].astype(dtype), y[perm].copy(), g, C,
                   f"mixture_n{n}_m{m}_s{seed}")


def clustered_mixture(n: int, m: int, seed: int, gamma: float, C: float = 1.0, comps: int = 3,
                      sigma: float = 0.7) -> Problem:
    """The mixture above with its rows grouped by component (class, then
    component), so that points that are near share 128-row tiles: the input
    order under which a narrow kernel leaves whole tiles near zero."""
    rng = np.random.default_rng(seed)
    y = _labels(n)
    means = rng.standard_normal((2, comps, m))
    cls = (y < 0).astype(np.int64)
    comp = rng.integers(0, comps, size=n)
    X = means[cls, comp] + sigma * rng.standard_normal((n, m))
    order = np.lexsort((rng.random(n), comp, cls))
    return Problem(X[order].astype(np.float32), y[order].copy(), gamma, C,
                   f"clustered_n{n}_m{m}_s{seed}")


# The five workloads, by what they are.
def plain_small() -> Problem:
    """n=1000, m=10 FP64 two-Gaussian set, gamma=1/m, C=1 (seed 0)."""
    return two_gaussians(1000, 10, seed=0)


def plain_large() -> Problem:
    """n=20000, m=128 FP32 3-component mixture, gamma=1/128, C=10 (seed 1)."""
    return mixture(20000, 128, seed=1, gamma=1.0 / 128, C=10.0)


def precision_large() -> Problem:
    """n=100000, m=64 FP32 mixture, gamma=0.5/64, C=1 (seed 2)."""
    return mixture(100000, 64, seed=2, gamma=0.5 / 64, C=1.0)


def batch_grid(datasets: int = 32, seed0: int = 100,
               Cs=(0.1, 1.0, 10.0, 100.0), gammas=(0.1, 0.5, 1.0, 2.0),
               n_lo: int = 200, n_hi: int = 4000, ms=(8, 32, 128, 256)):
    """`datasets` mixture sets x a C x gamma/m grid -> list of Problem.

    The features of one data set are shared (same array object) by its grid
    points, so a solver can reuse the Gram matrix across them.
    """
    out = []
    for d in range(datasets):
        rng = np.random.default_rng(seed0 + d)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(ms[rng.integers(0, len(ms))])
        base = mixture(n, m, seed=seed0 + d)
        for C in Cs:
            for g in gammas:
                out.append(Problem(base.X, base.y, g / m, C,
                                   f"grid_d{d}_C{C}_g{g}"))
    return out


@dataclasses.dataclass
class Request:
    t_arrive: float
    n: int
    m: int
    C: float
    seed: int


def poisson_requests(rate: float = 200.0, duration: float = 60.0, seed: int = 7,
                     n_lo: int = 500, n_hi: int = 50000, m_lo: int = 16, m_hi: int = 512,
                     C_lo: float = 0.1, C_hi: float = 100.0):
    """Arrival times (Poisson process) and shapes of SVM training requests."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        C = float(math.exp(rng.uniform(math.log(C_lo), math.log(C_hi))))
        out.append(Request(t, n, m, C, seed * 1000003 + k))
        k += 1
    return out


def request_problem(r: Request) -> Problem:
    """Materialise the training set of one request (gamma = 1/m)."""
    return mixture(r.n, r.m, seed=r.seed, gamma=1.0 / r.m, C=r.C)


def test_points(p: Problem, t: int, seed: int) -> np.ndarray:
    """Held-out points drawn like the training rows (perturbed copies)."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, p.n, size=t)
    Xt = p.X[idx].astype(np.float64) + 0.5 * rng.standard_normal((t, p.m))
    return Xt.astype(p.X.dtype)


def krr_targets(p: Problem, seed: int, noise: float = 0.1) -> np.ndarray:
    """Real targets t_i = sin(<w, x_i>) + noise * N(0, 1) with w ~ N(0, I/m):
    a smooth function of the features for the regression task (float32)."""
    rng = np.random.default_rng(seed)
    X = np.asarray(p.X, dtype=np.float64)
    w = rng.standard_normal(X.shape[1]) / math.sqrt(X.shape[1])
    t = np.sin(X @ w) + noise * rng.standard_normal(X.shape[0])
    return t.astype(np.float32)
