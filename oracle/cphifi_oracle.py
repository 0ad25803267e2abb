"""Plain FP64 NumPy oracle for the unaligned infinite-dimensional subproblem.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg, never by the library.  It is deliberately
slow and literal; every function names the passage of Brust & Kolda, "Fast and
Accurate CP-HIFI Tensor Decompositions Exploiting Kronecker Structure"
(arXiv 2603.25691) that it follows.

Conventions (Table 1 of the paper): ``n`` kernel-mode size, ``r`` rank,
``q`` observations, ``M`` product of the other mode sizes.  ``vec`` stacks
columns, so an n x r matrix X has ``vec(X)[i + n*j] = X[i, j]``.  Other-mode
indices are 0-based; the linear other-mode index is ``m = i_1 + n_1 (i_2 +
n_2 (...))`` (first other mode fastest), matching the Khatri-Rao ordering
``Z = A_d (.) ... (.) A_1`` of the mode-k unfolding (Appendix A.3).

The oracle solves the symmetric rho-regularised system of §4.1
(Eq. unaligned-infinite-1)::

    [F'F + lam (I_r (x) K) + rho I_rn] vec(W) = vec(K B)

Parity status of each function (what pins it in ``tests/test_oracle_*.py``):

* zhat, khatri_rao_rows, unfolding: brute-force Kruskal tensor + mode-k
  unfolding identity (Appendix A.3).
* F_matrix, system_matrix_*: literal S'(Z (x) K) with an explicit selection
  matrix; symmetry / positive-definiteness invariants.
* rhs_vec: equals F' t because S S' vec(T) = vec(T) (§2).
* solve_direct: zero gradient of the §2 objective by finite differences; the
  aligned closed form of Eq. W-decoupled (§3.2); NumPy least squares on the
  stacked least-squares form; a scalar closed form.
* matvec: dense system matrix; the one-step form below Eq. vl (§4.4.1).
* segment_grams, yhat1_from_grams, matvec_grams: the diagonal blocks of H in
  F'F = (I (x) K) H (I (x) K) assembled from the literal F; yhat1_from_grams
  against scatter_rows(gather_dot(..)) on tiny inputs.
* relative_residual: ||A d|| / ||b|| for W = W* + d with A and b assembled
  from the literal F (a wrong W must give a large residual), with the
  observations split into chunks that do not divide q.
* gram: explicit Khatri-Rao Z'Z.
* precond_apply: M^{-1}(M x) = x with M assembled from Eq. precon.
* pcg / cg: convergence to solve_direct; one iteration in the aligned case.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

__all__ = [
    "zhat", "khatri_rao_rows", "mttkrp", "rhs_vec", "gram", "F_matrix",
    "system_matrix_from_F", "system_matrix_blocks", "solve_direct",
    "kernel_times", "gather_dot", "scatter_rows", "matvec",
    "precond_setup", "precond_apply", "pcg", "cg", "relative_residual",
    "fitted_values", "vec", "unvec", "density", "segment_grams", "yhat1_from_grams",
    "matvec_grams", "fitted_error_sq_grams",
]


def vec(X: np.ndarray) -> np.ndarray:
    """Column-stacking vectorisation (Appendix A)."""
    return np.asarray(X, dtype=np.float64).reshape(-1, order="F")


def unvec(x: np.ndarray, n: int, r: int) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).reshape((n, r), order="F")


def density(n: int, other_sizes, q: int) -> float:
    """gamma = q / N with N the number of entries of the unfolding (§4.4.2)."""
    return q / (n * float(np.prod(other_sizes)))


# ---------------------------------------------------------------- §4.2 ----
def zhat(factors, oidx) -> np.ndarray:
    """Eq. zhat: row l of Zhat is the Hadamard product of the other modes'
    factor rows at observation l's other-mode indices."""
    q = oidx.shape[0]
    r = factors[0].shape[1]
    Z = np.ones((q, r))
    for c, A in enumerate(factors):
        Z = Z * np.asarray(A, dtype=np.float64)[oidx[:, c], :]
    return Z


def khatri_rao_rows(factors) -> np.ndarray:
    """Full Khatri-Rao product Z = A_d (.) ... (.) A_1 (M x r), built column by
    column from Kronecker products (Appendix A.1).  Only for tiny sizes."""
    r = factors[0].shape[1]
    cols = []
    for j in range(r):
        col = np.ones(1)
        for A in factors:               # A_1 first => it varies fastest
            col = np.kron(np.asarray(A, dtype=np.float64)[:, j], col)
        cols.append(col)
    return np.stack(cols, axis=1)


def F_matrix(K, kidx, Zh) -> np.ndarray:
    """Eq. F: F(l,:) = Zhat(l,:) (x) Khat(l,:) with Khat(l,:) = K(i_l,:)
    (Eq. khat).  q x nr, tiny sizes only."""
    K = np.asarray(K, dtype=np.float64)
    return np.stack([np.kron(Zh[l], K[kidx[l]]) for l in range(Zh.shape[0])]) \
        if Zh.shape[0] else np.zeros((0, K.shape[0] * Zh.shape[1]))


def mttkrp(n: int, kidx, vals, Zh) -> np.ndarray:
    """Sparse MTTKRP B = T Z (§4, below Eq. unaligned-infinite): row i of B is
    the sum over observations l with i_l = i of t_l * Zhat(l,:)."""
    r = Zh.shape[1]
    B = np.zeros((n, r))
    w = np.asarray(vals, dtype=np.float64)
    for j in range(r):
        B[:, j] = np.bincount(kidx, weights=w * Zh[:, j], minlength=n)
    return B


def rhs_vec(K, B) -> np.ndarray:
    """Right-hand side vec(K B) of Eq. unaligned-infinite-1."""
    return vec(np.asarray(K, dtype=np.float64) @ B)


def gram(factors) -> np.ndarray:
    """V = Z'Z computed as the Hadamard product of the factor Grams
    A_m' A_m (§3, after Eq. aligned-solve)."""
    r = factors[0].shape[1]
    V = np.ones((r, r))
    for A in factors:
        A = np.asarray(A, dtype=np.float64)
        V = V * (A.T @ A)
    return V


# ---------------------------------------------------------------- §4.1 ----
def system_matrix_from_F(F, K, lam: float, rho: float) -> np.ndarray:
    """F'F + lam (I_r (x) K) + rho I (Eq. unaligned-infinite-1)."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    r = F.shape[1] // n
    return F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)


def system_matrix_blocks(K, kidx, Zh, lam: float, rho: float) -> np.ndarray:
    """The same matrix without forming F.  Since F(l,:) = Zhat(l,:) (x) e_{i_l}'K,
    F'F = (I_r (x) K) H (I_r (x) K) with H = sum_l (Zhat(l,:)'Zhat(l,:)) (x)
    e_{i_l} e_{i_l}' (mixed-product rule, Appendix A.2)."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    r = Zh.shape[1]
    H = np.zeros((r, n, r, n))
    for i in range(n):
        rows = Zh[kidx == i]
        H[:, i, :, i] = rows.T @ rows
    H = H.reshape(r * n, r * n)        # index j*n + i  == vec order
    IK = np.kron(np.eye(r), K)
    return IK @ H @ IK + lam * IK + rho * np.eye(n * r)


def solve_direct(K, factors, kidx, oidx, vals, lam: float, rho: float,
                 use_F: bool | None = None) -> np.ndarray:
    """Direct solve of Eq. unaligned-infinite-1 by Cholesky (§4.1-§4.2).
    Returns W (n x r)."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    Zh = zhat(factors, oidx)
    r = Zh.shape[1]
    if use_F is None:
        use_F = Zh.shape[0] * n * r <= 4_000_000
    A = (system_matrix_from_F(F_matrix(K, kidx, Zh), K, lam, rho) if use_F
         else system_matrix_blocks(K, kidx, Zh, lam, rho))
    b = rhs_vec(K, mttkrp(n, kidx, vals, Zh))
    c = scipy.linalg.cho_factor(A, lower=True)
    return unvec(scipy.linalg.cho_solve(c, b), n, r)


# -------------------------------------------------------------- §4.4.1 ----
def kernel_times(K, X) -> np.ndarray:
    """Xhat = K X (first step of the matrix-free product)."""
    return np.asarray(K, dtype=np.float64) @ X


def gather_dot(Xh, kidx, Zh) -> np.ndarray:
    """Eq. vl: xbar_l = Xhat(i_l,:) . Zhat(l,:)."""
    return np.einsum("lr,lr->l", Xh[kidx], Zh)


def scatter_rows(n: int, kidx, xbar, Zh) -> np.ndarray:
    """Eq. yhat1: Yhat1(i,:) = sum over l with i_l = i of xbar_l Zhat(l,:)."""
    r = Zh.shape[1]
    Y = np.zeros((n, r))
    for j in range(r):
        Y[:, j] = np.bincount(kidx, weights=xbar * Zh[:, j], minlength=n)
    return Y


def matvec(K, kidx, Zh, lam: float, rho: float, X, chunk: int = 1 << 21):
    """y = (F'F + lam (I (x) K) + rho I) x in the four steps of §4.4.1:
    Xhat = K X; xbar_l = Xhat(i_l,:).Zhat(l,:); Yhat1 = sum_l xbar_l Zhat(l,:);
    Y = K Yhat1 + lam Xhat + rho X.

    Observations are visited in blocks of ``chunk`` purely to bound memory;
    the sum over l in Eq. yhat1 is the same sum."""
    K = np.asarray(K, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = K.shape[0]
    Xh = kernel_times(K, X)
    Y1 = np.zeros_like(X)
    q = kidx.shape[0]
    for s in range(0, q, chunk):
        e = min(q, s + chunk)
        Zc = np.asarray(Zh[s:e], dtype=np.float64)
        xb = gather_dot(Xh, kidx[s:e], Zc)
        Y1 += scatter_rows(n, kidx[s:e], xb, Zc)
    return K @ Y1 + lam * Xh + rho * X


def segment_grams(n: int, kidx, Zh, C=None) -> np.ndarray:
    """The per-index Gram blocks behind Eq. yhat1 (§4.4.1).  Row i of Yhat1
    only collects observations with i_l = i, and each adds
    (Xhat(i,:).Zhat(l,:)) Zhat(l,:) = (Zhat(l,:)' Zhat(l,:)) Xhat(i,:)', so
    Yhat1(i,:)' = C_i Xhat(i,:)' with C_i = sum over l with i_l = i of
    Zhat(l,:)' Zhat(l,:) (r x r).  These are the diagonal blocks of H in
    F'F = (I (x) K) H (I (x) K) (see system_matrix_blocks).  Returns an
    (n, r, r) array; with C given, the observations are added into it (so a
    long list can be visited in chunks)."""
    r = Zh.shape[1]
    if C is None:
        C = np.zeros((n, r, r))
    kidx = np.asarray(kidx)
    order = np.argsort(kidx, kind="stable")
    ks = kidx[order]
    bounds = np.searchsorted(ks, np.arange(n + 1))
    for i in np.unique(ks):
        rows = np.asarray(Zh[order[bounds[i]:bounds[i + 1]]], dtype=np.float64)
        C[i] += rows.T @ rows
    return C


def yhat1_from_grams(C, Xh) -> np.ndarray:
    """Eq. yhat1 through the per-index Gram blocks: Yhat1(i,:) = C_i Xhat(i,:)'
    (segment_grams)."""
    return np.einsum("ijk,ik->ij", C, np.asarray(Xh, dtype=np.float64))


def matvec_grams(K, C, lam: float, rho: float, X) -> np.ndarray:
    """The product of §4.4.1 with the gather-dot/scatter replaced by the
    per-index Gram blocks: y = K Yhat1 + lam Xhat + rho X, Xhat = K X,
    Yhat1(i,:) = C_i Xhat(i,:)'."""
    K = np.asarray(K, dtype=np.float64)
    Xh = kernel_times(K, X)
    return K @ yhat1_from_grams(C, Xh) + lam * Xh + rho * np.asarray(X, dtype=np.float64)


def fitted_error_sq_grams(K, C, E) -> float:
    """||F vec(E)||^2 = vec(E)' F'F vec(E) = sum_i (K E)(i,:) C_i (K E)(i,:)'
    (F'F = (I (x) K) H (I (x) K) with the blocks C_i of H)."""
    KE = kernel_times(K, E)
    return float(np.einsum("ij,ij->", KE, yhat1_from_grams(C, KE)))


def fitted_values(K, W, kidx, Zh) -> np.ndarray:
    """F vec(W): the model value at every observation, (K W)(i_l,:).Zhat(l,:)."""
    return gather_dot(kernel_times(K, W), kidx, Zh)


# -------------------------------------------------------------- §4.4.2 ----
def precond_setup(K, V, gamma: float, lam: float, rho: float, eigK=None):
    """Eigendecompositions (Eqs. eigK, eigV) and the n x r matrix D with
    D(i,j) = 1 / (gamma D_V(j) D_K(i)^2 + lam D_K(i) + rho) (Eq. fx and the
    definition of d above it).  Negative round-off eigenvalues of the PSD
    matrices are clamped to zero inside D only.  eigK = (D_K, U_K) from
    numpy.linalg.eigh(K) may be passed when it is already at hand."""
    dK, UK = eigK if eigK is not None else np.linalg.eigh(np.asarray(K, dtype=np.float64))
    dV, UV = np.linalg.eigh(np.asarray(V, dtype=np.float64))
    dK = np.maximum(dK, 0.0)
    dV = np.maximum(dV, 0.0)
    D = 1.0 / (gamma * np.outer(dK * dK, dV) + lam * dK[:, None] + rho)
    return UK, UV, D


def precond_apply(UK, UV, D, X) -> np.ndarray:
    """Eq. fx: M^{-1} x = U_K ((U_K' X U_V) o D) U_V'."""
    return UK @ ((UK.T @ X @ UV) * D) @ UV.T


# ----------------------------------------------------------- PCG (§4.4) ---
def pcg(apply_A, b, apply_Minv=None, tol: float = 1e-10, maxit: int = 1000,
        x0=None):
    """Preconditioned conjugate gradients (Golub & Van Loan, Matrix
    Computations, 4th ed., §11.5), written on n x r matrices with the
    Frobenius inner product (= the vec inner product).  Stops when the
    recurrence residual satisfies ||r||/||b|| <= tol or after maxit steps.
    Returns (X, iterations, list of relative residuals)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb if nb > 0 else 0.0]
    if nb == 0.0:
        return np.zeros_like(b), 0, hist
    k = 0
    p = None
    rz_old = None
    while hist[-1] > tol and k < maxit:
        z = apply_Minv(r) if apply_Minv is not None else r
        rz = float(np.sum(r * z))
        p = z.copy() if k == 0 else z + (rz / rz_old) * p
        Ap = apply_A(p)
        alpha = rz / float(np.sum(p * Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rz_old = rz
        k += 1
        hist.append(np.linalg.norm(r) / nb)
    return x, k, hist


def cg(apply_A, b, tol: float = 1e-10, maxit: int = 1000, x0=None):
    """Unpreconditioned CG (the 'cg' comparison of §5.2)."""
    return pcg(apply_A, b, None, tol, maxit, x0)


def relative_residual(K, factors, kidx, oidx, vals, lam, rho, W,
                      Zh=None, chunk: int = 1 << 21) -> float:
    """||b - A vec(W)|| / ||b|| for Eq. unaligned-infinite-1, in FP64."""
    K = np.asarray(K, dtype=np.float64)
    if Zh is None:
        Zh = zhat(factors, oidx)
    n = K.shape[0]
    B = np.zeros((n, Zh.shape[1]))
    q = kidx.shape[0]
    for s in range(0, q, chunk):
        e = min(q, s + chunk)
        B += mttkrp(n, kidx[s:e], vals[s:e], np.asarray(Zh[s:e], dtype=np.float64))
    b = K @ B
    R = b - matvec(K, kidx, Zh, lam, rho, np.asarray(W, dtype=np.float64), chunk)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(R) / nb) if nb > 0 else float(np.linalg.norm(R))
