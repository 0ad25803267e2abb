"""Plain FP64 oracle of the CP-HIFI alternating fit around the kernel-mode solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU legs,
never by the library.  Slow and literal; every function names the passage of
Brust & Kolda (arXiv 2603.25691) it follows.

The model (§2): a rank-r CP tensor whose kernel-mode factor is A_k = K W
(K the kernel matrix, W the weights) and whose other (finite) modes have
plain factor matrices A_m.  The fit minimises (§2 objective, with the rho
ridge of §4.1 on W)

    J = sum_{l in Omega} (t_l - m_l)^2 + lam vec(W)'(I_r (x) K) vec(W) + rho ||W||^2,
    m_l = sum_j (K W)(i_l, j) prod_m A_m(i_m^l, j),

alternating over the modes (§2, Eq. cp-hifi-subproblem): the kernel mode is
the subproblem of §4 (solved here directly, or by the GPU's PCG), a finite
mode has no regulariser (R_m = 0, §2) and its update is the CP-ALS step for
incomplete data: each row i of A_m solves its own r x r normal equations
over the observations with i_m = i.  The paper does not spell that step out
(it cites it as known); the reading used here adds a ridge of 1e-12 trace(G)
to rows with fewer than r observations and leaves rows with no observation
(or an all-zero Gram) unchanged.

Parity status (``tests/test_oracle_als_pins.py``): model_values against a
brute-force dense Kruskal tensor; finite_update by the zero gradient of J in
A_m (central differences), exact recovery of planted noise-free factors, and
a planted mistake that must fail; als by a non-increasing objective.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import cphifi_oracle as _k

__all__ = ["kernel_factor", "model_values", "objective", "fit_error", "finite_update",
           "kernel_update", "als"]


def kernel_factor(K, W) -> np.ndarray:
    """A_k = K_k W_k (§2): the kernel-mode factor of the model."""
    return np.asarray(K, dtype=np.float64) @ np.asarray(W, dtype=np.float64)


def model_values(K, W, factors, kidx, oidx) -> np.ndarray:
    """m_l = sum_j A_k(i_l, j) prod_m A_m(i_m^l, j): the CP model at the
    observed entries (the Kruskal tensor of §2, read at Omega)."""
    prod = kernel_factor(K, W)[kidx]
    for m, F in enumerate(factors):
        prod = prod * np.asarray(F, dtype=np.float64)[oidx[:, m]]
    return prod.sum(axis=1)


def objective(K, W, factors, kidx, oidx, vals, lam: float, rho: float) -> float:
    """J of the module docstring (§2 objective with the §4.1 ridge)."""
    res = np.asarray(vals, dtype=np.float64) - model_values(K, W, factors, kidx, oidx)
    W = np.asarray(W, dtype=np.float64)
    return float(res @ res + lam * np.sum(W * (np.asarray(K) @ W)) + rho * np.sum(W * W))


def fit_error(K, W, factors, kidx, oidx, vals) -> float:
    """Relative error of the fit at the observed entries, ||t - m|| / ||t||."""
    t = np.asarray(vals, dtype=np.float64)
    res = t - model_values(K, W, factors, kidx, oidx)
    nt = np.linalg.norm(t)
    return float(np.linalg.norm(res) / nt) if nt > 0 else float(np.linalg.norm(res))


def finite_update(K, W, factors, m: int, kidx, oidx, vals, ridge: float = 1e-12) -> np.ndarray:
    """New A_m for a finite mode m (§2: R_m = 0, the CP-ALS step).

    With z_l = A_k(i_l,:) o prod_{m' != m} A_m'(i_m'^l,:), row i of A_m
    minimises sum_{l: i_m^l = i} (t_l - a . z_l)^2, i.e. solves
    G_i a = h_i with G_i = sum z_l z_l', h_i = sum t_l z_l (Cholesky)."""
    Z = kernel_factor(K, W)[kidx]
    for m2, F in enumerate(factors):
        if m2 != m:
            Z = Z * np.asarray(F, dtype=np.float64)[oidx[:, m2]]
    t = np.asarray(vals, dtype=np.float64)
    old = np.asarray(factors[m], dtype=np.float64)
    new = old.copy()
    r = Z.shape[1]
    rows = oidx[:, m]
    for i in range(old.shape[0]):
        sel = rows == i
        cnt = int(sel.sum())
        if cnt == 0:
            continue
        Zi = Z[sel]
        G = Zi.T @ Zi
        tr = float(np.trace(G))
        if tr == 0.0:
            continue
        if cnt < r:
            G = G + ridge * tr * np.eye(r)
        h = Zi.T @ t[sel]
        c = scipy.linalg.cho_factor(G, lower=True)
        new[i] = scipy.linalg.cho_solve(c, h)
    return new


def kernel_update(K, factors, kidx, oidx, vals, lam: float, rho: float, W0=None,
                  method: str = "direct", tol: float = 1e-12, maxit: int = 5000) -> np.ndarray:
    """The kernel-mode subproblem of §4 (Eq. unaligned-infinite-1): the
    direct Cholesky solve, or PCG with the §4.4.2 preconditioner from W0."""
    if method == "direct":
        return _k.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    n = np.asarray(K).shape[0]
    Zh = _k.zhat(factors, oidx)
    b = _k.rhs_vec(K, _k.mttkrp(n, kidx, vals, Zh)).reshape(n, -1, order="F")
    g = _k.density(n, [F.shape[0] for F in factors], kidx.shape[0])
    UK, UV, D = _k.precond_setup(K, _k.gram(factors), g, lam, rho)
    W, _, _ = _k.pcg(lambda X: _k.matvec(K, kidx, Zh, lam, rho, X), b,
                     lambda R: _k.precond_apply(UK, UV, D, R), tol=tol, maxit=maxit, x0=W0)
    return W


def als(K, factors, kidx, oidx, vals, lam: float, rho: float, sweeps: int,
        tol: float = 0.0, W0=None, method: str = "direct"):
    """Alternating optimisation (§2): per sweep the kernel mode (§4, warm
    started from the previous W), then each finite mode in order; stops after
    `sweeps` sweeps or when the fit error changes by less than `tol` (§5:
    tolerance on the change in the ALS error).  Returns (W, factors, errors
    after each sweep, objectives after each sub-step)."""
    factors = [np.array(F, dtype=np.float64) for F in factors]
    W = None if W0 is None else np.array(W0, dtype=np.float64)
    errs, objs = [], []
    for _ in range(sweeps):
        W = kernel_update(K, factors, kidx, oidx, vals, lam, rho, W0=W, method=method)
        objs.append(objective(K, W, factors, kidx, oidx, vals, lam, rho))
        for m in range(len(factors)):
            factors[m] = finite_update(K, W, factors, m, kidx, oidx, vals)
            objs.append(objective(K, W, factors, kidx, oidx, vals, lam, rho))
        errs.append(fit_error(K, W, factors, kidx, oidx, vals))
        if tol > 0 and len(errs) > 1 and abs(errs[-2] - errs[-1]) < tol:
            break
    return W, factors, errs, objs
