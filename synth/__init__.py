"""Seeded synthetic inputs for the unaligned kernel-mode subproblem.

This module only *draws data*: design points, kernel matrices, finite-mode
factors, observation index lists and planted observation values.  It holds
none of the solver's arithmetic (no Khatri-Rao rows, no right-hand side, no
operator, no preconditioner) and is shared by the FP64 oracle, the tests and
the benchmark so that both sides of every parity check see identical inputs.

Recipe (the paper's own datasets are not available, so these stand in for
them; §5 describes the real data, §4 the subproblem):

* design points: ``x_i = i/(n-1)`` on [0, 1] (the paper's grids are evenly
  spaced, §5.1), or integer coordinates ``1..n`` for the paper-shaped runs;
* kernel: Gaussian ``exp(-(x-y)^2 / (2 sigma^2))`` or Matern-3/2
  ``(1 + sqrt(3) d/ell) exp(-sqrt(3) d/ell)``;
* finite-mode factors: i.i.d. N(0, 1);
* observations: ``q`` entries drawn uniformly without replacement from the
  ``n * M`` entries of the mode-k unfolding, returned sorted by
  (kernel index, other-mode linear index) unless ``shuffle=True``;
* values: planted smooth CP model
  ``T(i, i_1, .., i_d) = sum_j f_j(x_i) prod_m A_m(i_m, j) + eps`` with
  ``f_j(x) = a_j sin(2 pi w_j x) + b_j cos(2 pi w'_j x)``, ``w ~ U[1, 4]``,
  ``a, b ~ N(0, 1)`` and ``eps = noise * rms(T_Omega) * N(0, 1)``.
"""
from __future__ import annotations

import dataclasses
import numpy as np


def grid_points(n: int, integer: bool = False) -> np.ndarray:
    if integer:
        return np.arange(1, n + 1, dtype=np.float64)
    if n == 1:
        return np.zeros(1)
    return np.arange(n, dtype=np.float64) / (n - 1)


def gaussian_kernel(x: np.ndarray, sigma: float) -> np.ndarray:
    d = x[:, None] - x[None, :]
    return np.exp(-(d * d) / (2.0 * sigma * sigma))


def matern32_kernel(x: np.ndarray, ell: float) -> np.ndarray:
    d = np.abs(x[:, None] - x[None, :]) * (np.sqrt(3.0) / ell)
    return (1.0 + d) * np.exp(-d)


@dataclasses.dataclass
class Problem:
    """One unaligned kernel-mode subproblem (all arrays host numpy).

    K        (n, n) float64, symmetric PSD kernel matrix
    factors  list of (n_m, r) float64 finite-mode factors, m = 1..d_other
    kidx     (q,) int32 kernel-mode index of each observation
    oidx     (q, d_other) int32 other-mode indices of each observation
    vals     (q,) float64 observed values
    lam, rho regularisation parameters
    """
    K: np.ndarray
    factors: list
    kidx: np.ndarray
    oidx: np.ndarray
    vals: np.ndarray
    lam: float
    rho: float
    x: np.ndarray = None

    @property
    def n(self) -> int:
        return self.K.shape[0]

    @property
    def r(self) -> int:
        return self.factors[0].shape[1]

    @property
    def q(self) -> int:
        return int(self.kidx.shape[0])

    @property
    def other_sizes(self) -> list:
        return [int(a.shape[0]) for a in self.factors]


def sample_observations(rng: np.random.Generator, n: int, other_sizes, q: int,
                        shuffle: bool = False):
    """Draw q distinct entries of the n x M unfolding, uniformly.

    The linear index is ``i * M + m`` with ``m = i_1 + n_1 (i_2 + n_2 (...))``
    (first other mode fastest), so sorting it sorts by kernel index first.
    """
    M = int(np.prod(other_sizes))
    total = n * M
    if q > total:
        raise ValueError("q exceeds the number of entries")
    if q == 0:
        lin = np.zeros(0, dtype=np.int64)
    elif q * 4 >= total:
        lin = np.sort(rng.choice(total, size=q, replace=False))
    else:
        # Bernoulli(p) sampling of the entries (geometric gaps, so the result
        # is sorted and distinct), with p a little above q/total, followed by
        # dropping a uniformly chosen surplus: every q-subset is equally likely.
        p = min(1.0, q / total * 1.02 + 8.0 / total + 4.0 * np.sqrt(q) / total)
        while True:
            gaps = rng.geometric(p, size=int(q * 1.05 + 6 * np.sqrt(q) + 64))
            lin = np.cumsum(gaps, dtype=np.int64) - 1
            lin = lin[lin < total]
            if lin.shape[0] >= q:
                break
            p = min(1.0, p * 1.05)
        if lin.shape[0] > q:
            keep = np.ones(lin.shape[0], dtype=bool)
            keep[rng.choice(lin.shape[0], size=lin.shape[0] - q, replace=False)] = False
            lin = lin[keep]
    if shuffle:
        lin = lin[rng.permutation(lin.shape[0])]
    kidx = (lin // M).astype(np.int32)
    m = lin % M
    oidx = np.empty((lin.shape[0], len(other_sizes)), dtype=np.int32)
    for c, nm in enumerate(other_sizes):
        oidx[:, c] = (m % nm).astype(np.int32)
        m = m // nm
    return kidx, oidx


def planted_values(rng: np.random.Generator, x: np.ndarray, factors, kidx, oidx,
                   noise: float, chunk: int = 1 << 22) -> np.ndarray:
    """Evaluate the planted smooth CP model at the observed entries."""
    r = factors[0].shape[1]
    w1 = rng.uniform(1.0, 4.0, size=r)
    w2 = rng.uniform(1.0, 4.0, size=r)
    a = rng.standard_normal(r)
    b = rng.standard_normal(r)
    fx = a * np.sin(2 * np.pi * np.outer(x, w1)) + b * np.cos(2 * np.pi * np.outer(x, w2))
    q = kidx.shape[0]
    vals = np.empty(q, dtype=np.float64)
    if len(factors) == 2 and q > (1 << 22) and np.all(np.diff(kidx) >= 0):
        # Large sorted two-mode case: per kernel index, the full n_1 x n_2
        # slice of the planted model is one small matrix product.
        A1, A2 = factors
        bounds = np.searchsorted(kidx, np.arange(x.shape[0] + 1))
        for i in range(x.shape[0]):
            s, e = bounds[i], bounds[i + 1]
            if s == e:
                continue
            G = (A1 * fx[i]) @ A2.T
            vals[s:e] = G[oidx[s:e, 0], oidx[s:e, 1]]
    else:
        for s in range(0, q, chunk):
            e = min(q, s + chunk)
            prod = fx[kidx[s:e]]
            for c, A in enumerate(factors):
                prod = prod * A[oidx[s:e, c]]
            vals[s:e] = prod.sum(axis=1)
    if q:
        rms = float(np.sqrt(np.mean(vals * vals)))
        vals += noise * rms * rng.standard_normal(q)
    return vals


def planted_problem(seed: int, n: int, other_sizes, q: int, r: int, *,
                    kernel: str = "gaussian", bandwidth: float = 0.1,
                    integer_grid: bool = False, lam: float = 1e-4,
                    rho: float = 1e-6, noise: float = 0.01,
                    shuffle: bool = False, aligned: bool = False) -> Problem:
    """A planted-low-rank unaligned subproblem (see the module docstring).

    ``aligned=True`` observes every entry of the unfolding (q = n*M), the
    special case in which the system decouples.
    """
    rng = np.random.default_rng(seed)
    x = grid_points(n, integer_grid)
    if kernel == "gaussian":
        K = gaussian_kernel(x, bandwidth)
    elif kernel == "matern32":
        K = matern32_kernel(x, bandwidth)
    else:
        raise ValueError(kernel)
    factors = [rng.standard_normal((nm, r)) for nm in other_sizes]
    if aligned:
        q = n * int(np.prod(other_sizes))
    kidx, oidx = sample_observations(rng, n, other_sizes, q, shuffle=shuffle)
    vals = planted_values(rng, x, factors, kidx, oidx, noise)
    return Problem(K=K, factors=factors, kidx=kidx, oidx=oidx, vals=vals,
                   lam=lam, rho=rho, x=x)


# Named workloads (sizes from the subproblem configurations this library is
# measured on).  ``tiny`` shapes are for brute-force checks.
WORKLOADS = {
    # n=100 Gaussian sigma=0.1, finite 20x30, q=6000 (10%), r=5, lambda=1e-4
    "c1_fp64_n100_q6e3_r5": dict(n=100, other_sizes=(20, 30), q=6000, r=5,
                                 bandwidth=0.1, lam=1e-4, rho=1e-6),
    # n=8000, finite 400x500, q=5e7, r=40 (mixed precision single solve)
    "c3_mixed_n8000_q5e7_r40": dict(n=8000, other_sizes=(400, 500), q=50_000_000,
                                    r=40, bandwidth=0.1, lam=1e-4, rho=1e-6),
    # kernel-mode solve of the alternating fit: n=2000, 200x300, q=6e6, r=20
    "c2_fp64_n2000_q6e6_r20": dict(n=2000, other_sizes=(200, 300), q=6_000_000,
                                   r=20, bandwidth=0.1, lam=1e-4, rho=1e-6),
}


# Kernel sizes of the batched / served streams: n is drawn log-uniform on
# [50, 2000] and snapped to this 16-point log grid, so that kernels (and their
# one-time eigendecompositions) are shared between instances, as the kernel
# mode of one tensor is across ALS sweeps.
BATCH_N_GRID = tuple(int(round(50 * (40.0 ** (k / 15.0)))) for k in range(16))


def batch_specs(seed: int, count: int = 256):
    """Instance shapes of a batch of uneven kernel-mode subproblems.

    n ~ logU[50, 2000] (snapped to BATCH_N_GRID), M ~ logU[100, 5e4] split into
    two finite modes of about sqrt(M) rows each, q ~ logU[1e3, 1e6] capped at
    floor(0.5 n M), r uniform in {4, 8, 16, 32}, Gaussian or Matern-3/2 kernel
    (bandwidth 0.1) with probability 1/2 each.  Returns a list of dicts with
    keys n, other_sizes, q, r, kernel, seed.
    """
    rng = np.random.default_rng(seed)
    grid = np.array(BATCH_N_GRID, dtype=np.float64)
    out = []
    for k in range(count):
        n_raw = np.exp(rng.uniform(np.log(50.0), np.log(2000.0)))
        n = int(grid[np.argmin(np.abs(np.log(grid) - np.log(n_raw)))])
        M = np.exp(rng.uniform(np.log(100.0), np.log(5e4)))
        n1 = max(1, int(round(np.sqrt(M))))
        n2 = max(1, int(round(M / n1)))
        q = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e6)))))
        q = min(q, (n * n1 * n2) // 2)
        r = int(rng.choice([4, 8, 16, 32]))
        kernel = "gaussian" if rng.uniform() < 0.5 else "matern32"
        out.append(dict(n=n, other_sizes=(n1, n2), q=q, r=r, kernel=kernel,
                        seed=int(rng.integers(1 << 31))))
    return out


def batch_problem(spec: dict, lam: float = 1e-4, rho: float = 1e-6) -> Problem:
    """The planted subproblem of one batch_specs entry (sorted observations)."""
    return planted_problem(spec["seed"], spec["n"], spec["other_sizes"], spec["q"],
                           spec["r"], kernel=spec["kernel"], bandwidth=0.1, lam=lam,
                           rho=rho)


def workload(name: str, seed: int = 0, **over) -> Problem:
    kw = dict(WORKLOADS[name])
    kw.update(over)
    return planted_problem(seed, kw.pop("n"), kw.pop("other_sizes"), kw.pop("q"),
                           kw.pop("r"), **kw)
