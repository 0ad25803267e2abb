"""Pins of the FP64 oracle against facts that do not come from the oracle.

Every check here compares the oracle with something fixed by the paper or by
mathematics: brute-force assembly from the problem statement (explicit
selection matrix S and Kronecker product Z (x) K, §2), the Kruskal-tensor
unfolding identity (Appendix A.3), the aligned closed form (Eq. W-decoupled,
§3.2), the dense preconditioner of Eq. precon (§4.4.2), finite differences of
the §2 objective, NumPy least squares on the stacked problem, hand-derived
fixtures in ``tests/golden/`` and invariants (symmetry, definiteness).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import oracle.cphifi_oracle as OC
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_problem(seed=0, n=4, other=(2, 3), q=11, r=2, lam=0.3, rho=0.05,
                 sigma=0.4, aligned=False):
    rng = np.random.default_rng(seed)
    x = synth.grid_points(n)
    K = synth.gaussian_kernel(x, sigma)
    factors = [rng.standard_normal((nm, r)) for nm in other]
    if aligned:
        q = n * int(np.prod(other))
    kidx, oidx = synth.sample_observations(rng, n, other, q, shuffle=True)
    vals = rng.standard_normal(q)
    return K, factors, kidx, oidx, vals, lam, rho


def linear_other_index(oidx, other):
    m = np.zeros(oidx.shape[0], dtype=np.int64)
    stride = 1
    for c, nm in enumerate(other):
        m += oidx[:, c].astype(np.int64) * stride
        stride *= nm
    return m


def selection_matrix(n, M, kidx, m):
    """S (nM x q): column l selects entry (i_l, m_l) of vec(T), index i + n m."""
    S = np.zeros((n * M, kidx.shape[0]))
    S[kidx + n * m, np.arange(kidx.shape[0])] = 1.0
    return S


def literal_F(K, factors, kidx, oidx):
    """F = S'(Z (x) K) straight from §2 / Eq. unaligned-infinite."""
    other = [a.shape[0] for a in factors]
    n, M = K.shape[0], int(np.prod(other))
    Z = O.khatri_rao_rows(factors)
    S = selection_matrix(n, M, kidx, linear_other_index(oidx, other))
    return S.T @ np.kron(Z, K)


# --------------------------------------------------------------- Zhat / Z ---
def test_khatri_rao_matches_kruskal_unfolding():
    """Appendix A.3: the mode-k unfolding of a Kruskal tensor is A_k Z'."""
    rng = np.random.default_rng(1)
    n, other, r = 3, (2, 3, 2), 2
    A0 = rng.standard_normal((n, r))
    facs = [rng.standard_normal((nm, r)) for nm in other]
    T = np.zeros((n,) + other)
    for i in range(n):
        for a in range(other[0]):
            for b in range(other[1]):
                for c in range(other[2]):
                    T[i, a, b, c] = sum(A0[i, j] * facs[0][a, j] * facs[1][b, j]
                                        * facs[2][c, j] for j in range(r))
    # unfolding column index m = a + n1 (b + n2 c)  (first other mode fastest)
    Tk = T.reshape(n, -1, order="F")
    np.testing.assert_allclose(Tk, A0 @ O.khatri_rao_rows(facs).T, rtol=1e-13, atol=1e-13)


def test_zhat_rows_are_khatri_rao_rows():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(other=(2, 3, 2), q=9)
    Z = O.khatri_rao_rows(factors)
    m = linear_other_index(oidx, [a.shape[0] for a in factors])
    np.testing.assert_allclose(O.zhat(factors, oidx), Z[m], rtol=1e-14, atol=1e-14)


def test_gram_is_ZtZ():
    K, factors, *_ = tiny_problem(other=(3, 4, 2), r=3)
    Z = O.khatri_rao_rows(factors)
    np.testing.assert_allclose(O.gram(factors), Z.T @ Z, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------- F ---
def test_F_rows_equal_selected_kronecker_rows():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem()
    Zh = O.zhat(factors, oidx)
    np.testing.assert_allclose(O.F_matrix(K, kidx, Zh), literal_F(K, factors, kidx, oidx),
                               rtol=1e-13, atol=1e-14)


def test_rhs_equals_F_transpose_t():
    """b = vec(K B) = F't because S S' vec(T) = vec(T) (§2, §4.1)."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=17)
    Zh = O.zhat(factors, oidx)
    b = O.rhs_vec(K, O.mttkrp(K.shape[0], kidx, vals, Zh))
    np.testing.assert_allclose(b, literal_F(K, factors, kidx, oidx).T @ vals, rtol=1e-12, atol=1e-13)


def test_mttkrp_equals_dense_unfolding_times_Z():
    """B = T Z with T the zero-filled unfolding (§2 assumption S S' vec T = vec T)."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=13)
    other = [a.shape[0] for a in factors]
    n, M = K.shape[0], int(np.prod(other))
    T = np.zeros((n, M))
    T[kidx, linear_other_index(oidx, other)] = vals
    Zh = O.zhat(factors, oidx)
    np.testing.assert_allclose(O.mttkrp(n, kidx, vals, Zh), T @ O.khatri_rao_rows(factors),
                               rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------- system matrix ---
def test_block_assembly_equals_F_assembly():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=15, r=3)
    Zh = O.zhat(factors, oidx)
    A1 = O.system_matrix_from_F(O.F_matrix(K, kidx, Zh), K, lam, rho)
    A2 = O.system_matrix_blocks(K, kidx, Zh, lam, rho)
    np.testing.assert_allclose(A1, A2, rtol=1e-12, atol=1e-13)


def test_system_matrix_literal_and_invariants():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=14, r=2)
    n, r = K.shape[0], 2
    F = literal_F(K, factors, kidx, oidx)
    A_lit = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    A = O.system_matrix_from_F(O.F_matrix(K, kidx, O.zhat(factors, oidx)), K, lam, rho)
    np.testing.assert_allclose(A, A_lit, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13)
    # F'F and lam (I (x) K) are PSD, so every eigenvalue is at least rho (§4.1)
    assert np.linalg.eigvalsh(A).min() >= rho * (1 - 1e-8)


# ----------------------------------------------------------------- matvec ---
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matvec_equals_dense_system(seed):
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(seed=seed, n=5, q=19, r=3)
    n, r = K.shape[0], 3
    F = literal_F(K, factors, kidx, oidx)
    A_lit = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    X = np.random.default_rng(seed + 10).standard_normal((n, r))
    Y = O.matvec(K, kidx, O.zhat(factors, oidx), lam, rho, X, chunk=4)
    np.testing.assert_allclose(O.vec(Y), A_lit @ O.vec(X), rtol=1e-12, atol=1e-12)


def test_two_step_equals_one_step_form():
    """§4.4.1: v_l = K(i_l,:) X Zhat(l,:)' (one step) equals the two-step
    Xhat = K X, v_l = Xhat(i_l,:) Zhat(l,:)'."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=12, r=3)
    Zh = O.zhat(factors, oidx)
    X = np.random.default_rng(5).standard_normal((K.shape[0], 3))
    one_step = np.array([K[kidx[l], :] @ X @ Zh[l] for l in range(len(kidx))])
    np.testing.assert_allclose(O.gather_dot(O.kernel_times(K, X), kidx, Zh), one_step,
                               rtol=1e-13, atol=1e-13)
    # and F x equals the same vector (F = S'(Z (x) K))
    np.testing.assert_allclose(literal_F(K, factors, kidx, oidx) @ O.vec(X), one_step,
                               rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------ direct solve ---
def objective(w, F, t, K, lam, rho, r):
    """§2 subproblem objective with the §4.1 ridge: ||F w - t||^2 +
    lam w'(I (x) K) w + rho ||w||^2."""
    res = F @ w - t
    return res @ res + lam * w @ np.kron(np.eye(r), K) @ w + rho * w @ w


def test_direct_solution_zeroes_objective_gradient():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=16, r=2)
    n, r = K.shape[0], 2
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    F = literal_F(K, factors, kidx, oidx)
    w = O.vec(W)
    h = 1e-4
    g = np.array([(objective(w + h * e, F, vals, K, lam, rho, r)
                   - objective(w - h * e, F, vals, K, lam, rho, r)) / (2 * h)
                  for e in np.eye(n * r)])
    g0 = np.array([(objective(h * e, F, vals, K, lam, rho, r)
                    - objective(-h * e, F, vals, K, lam, rho, r)) / (2 * h)
                   for e in np.eye(n * r)])
    assert np.linalg.norm(g) <= 1e-8 * np.linalg.norm(g0)


def test_direct_matches_stacked_least_squares():
    """The minimiser of ||F w - t||^2 + lam ||(I (x) K^1/2) w||^2 + rho ||w||^2
    by NumPy's QR/SVD least squares on the stacked system."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=18, r=2, seed=3)
    n, r = K.shape[0], 2
    d, U = np.linalg.eigh(K)
    Khalf = (U * np.sqrt(np.maximum(d, 0))) @ U.T
    F = literal_F(K, factors, kidx, oidx)
    A = np.vstack([F, np.sqrt(lam) * np.kron(np.eye(r), Khalf), np.sqrt(rho) * np.eye(n * r)])
    rhs = np.concatenate([vals, np.zeros(2 * n * r)])
    w_ls = np.linalg.lstsq(A, rhs, rcond=None)[0]
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    np.testing.assert_allclose(O.vec(W), w_ls, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("rho", [0.0, 1e-3])
def test_aligned_case_closed_form(rho):
    """Aligned Omega (every entry observed): S S' = I, F'F = V (x) K^2 and the
    solution is U_K((U_K' K B U_V) o D') U_V' with
    D'(i,j) = 1/(D_V(j) D_K(i)^2 + lam D_K(i) + rho).  With rho = 0 and K
    positive definite this is exactly Eq. W-decoupled (§3.2),
    W = U_K((U_K' B U_V) o D)U_V', D(i,j) = 1/(D_V(j) D_K(i) + lam)."""
    n, other, r, lam = 5, (2, 3), 2, 0.2
    K, factors, kidx, oidx, vals, _, _ = tiny_problem(n=n, other=other, r=r, lam=lam,
                                                      sigma=0.15, aligned=True)
    M = int(np.prod(other))
    T = np.zeros((n, M))
    T[kidx, linear_other_index(oidx, other)] = vals
    Z = O.khatri_rao_rows(factors)
    B = T @ Z
    dK, UK = np.linalg.eigh(K)
    dV, UV = np.linalg.eigh(Z.T @ Z)
    assert dK.min() > 1e-3
    if rho == 0.0:
        Dm = 1.0 / (np.outer(dK, dV) + lam)
        W_cf = UK @ ((UK.T @ B @ UV) * Dm) @ UV.T
    else:
        Dm = 1.0 / (np.outer(dK ** 2, dV) + lam * dK[:, None] + rho)
        W_cf = UK @ ((UK.T @ K @ B @ UV) * Dm) @ UV.T
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    np.testing.assert_allclose(W, W_cf, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("name", ["scalar_case", "two_point_case"])
def test_hand_derived_fixtures(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    W = O.solve_direct(np.array(g["K"]), [np.array(g["factor"])],
                       np.array(g["kidx"], dtype=np.int32), np.array(g["oidx"], dtype=np.int32),
                       np.array(g["vals"]), g["lambda"], g["rho"])
    np.testing.assert_allclose(W, np.array(g["W"]), rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------- preconditioner ---
def test_precond_inverts_dense_eq_precon():
    """M = gamma (V (x) K^2) + lam (I (x) K) + rho I (Eq. precon); the
    eigen-form apply (Eq. fx) must invert it."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=10, r=3)
    n, r = K.shape[0], 3
    V = O.gram(factors)
    gamma = O.density(n, [a.shape[0] for a in factors], len(kidx))
    Mden = gamma * np.kron(V, K @ K) + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    UK, UV, D = O.precond_setup(K, V, gamma, lam, rho)
    X = np.random.default_rng(9).standard_normal((n, r))
    MX = O.unvec(Mden @ O.vec(X), n, r)
    np.testing.assert_allclose(O.precond_apply(UK, UV, D, MX), X, rtol=1e-8, atol=1e-9)


# ------------------------------------------------------------------ PCG/CG ---
def _operators(K, factors, kidx, oidx, vals, lam, rho):
    n = K.shape[0]
    Zh = O.zhat(factors, oidx)
    b = O.kernel_times(K, O.mttkrp(n, kidx, vals, Zh))
    V = O.gram(factors)
    gamma = O.density(n, [a.shape[0] for a in factors], len(kidx))
    UK, UV, D = O.precond_setup(K, V, gamma, lam, rho)
    return (lambda X: O.matvec(K, kidx, Zh, lam, rho, X), b,
            lambda R: O.precond_apply(UK, UV, D, R))


def test_pcg_one_iteration_when_aligned():
    """Aligned data: gamma = 1 and M = A, so PCG stops after one step (§4.4.2)."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(n=5, other=(2, 3), r=2,
                                                          aligned=True)
    A, b, Minv = _operators(K, factors, kidx, oidx, vals, lam, rho)
    X, it, hist = O.pcg(A, b, Minv, tol=1e-10, maxit=50)
    assert it == 1 and hist[-1] <= 1e-10
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    np.testing.assert_allclose(X, W, rtol=1e-8, atol=1e-10)


def test_pcg_and_cg_reach_direct_solution():
    p = synth.planted_problem(4, 12, (5, 6), 150, 3, bandwidth=0.15, lam=1e-2, rho=1e-2)
    A, b, Minv = _operators(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    W = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    Xp, itp, _ = O.pcg(A, b, Minv, tol=1e-12, maxit=500)
    Xc, itc, _ = O.cg(A, b, tol=1e-12, maxit=5000)
    np.testing.assert_allclose(Xp, W, rtol=1e-8, atol=1e-9 * np.abs(W).max())
    np.testing.assert_allclose(Xc, W, rtol=1e-8, atol=1e-9 * np.abs(W).max())
    assert itp < itc   # the preconditioner pays (§5.2: cg needs more iterations)


def test_pcg_c1_shape_residual_and_fit():
    """The n=100 / 20x30 / q=6000 / r=5 workload: PCG to 1e-10 matches the
    direct solve in the fitted values and has a tiny true residual."""
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=0)
    A, b, Minv = _operators(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    X, it, _ = O.pcg(A, b, Minv, tol=1e-10, maxit=500)
    W = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, X)
    assert res <= 1e-10 * 1.5
    Zh = O.zhat(p.factors, p.oidx)
    fx, fw = O.fitted_values(p.K, X, p.kidx, Zh), O.fitted_values(p.K, W, p.kidx, Zh)
    assert np.linalg.norm(fx - fw) <= 1e-8 * np.linalg.norm(fw)
    assert it < 100


def test_relative_residual_of_direct_solution_is_tiny():
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=15)
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    assert O.relative_residual(K, factors, kidx, oidx, vals, lam, rho, W) < 1e-12


@pytest.mark.parametrize("chunk", [4, 5, 1 << 21])
def test_relative_residual_of_a_wrong_W(chunk):
    """For W = W* + d the residual is A vec(d) (A W* = b), so the oracle must
    report ||A vec(d)|| / ||b|| with A and b assembled from the literal F
    (b = F't, §2 and §4.1).  q = 15 is not a multiple of the chunk sizes 4 and
    5, so the chunked sums over observations are covered too."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=15, r=2, seed=6)
    n, r = K.shape[0], 2
    F = literal_F(K, factors, kidx, oidx)
    A = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    b = F.T @ vals
    Ws = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho)
    rng = np.random.default_rng(7)
    for scale in (1.0, 1e-3, 1e-7):
        d = scale * rng.standard_normal((n, r))
        want = np.linalg.norm(A @ O.vec(d)) / np.linalg.norm(b)
        got = O.relative_residual(K, factors, kidx, oidx, vals, lam, rho, Ws + d, chunk=chunk)
        assert want > 1e-9
        np.testing.assert_allclose(got, want, rtol=1e-6)
    # the zero start has residual exactly 1
    z = O.relative_residual(K, factors, kidx, oidx, vals, lam, rho, np.zeros((n, r)),
                            chunk=chunk)
    np.testing.assert_allclose(z, 1.0, rtol=1e-13)


def test_relative_residual_catches_a_dropped_ridge(monkeypatch):
    """A residual routine that dropped the rho term would call a wrong W
    converged; the pin above must catch it (mistake planted in the oracle)."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=15, r=2, seed=6, rho=0.5)
    n, r = K.shape[0], 2
    F = literal_F(K, factors, kidx, oidx)
    A = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    b = F.T @ vals
    d = np.random.default_rng(8).standard_normal((n, r))
    W = O.solve_direct(K, factors, kidx, oidx, vals, lam, rho) + d
    want = np.linalg.norm(A @ O.vec(d)) / np.linalg.norm(b)
    good = OC.matvec
    monkeypatch.setattr(OC, "matvec", lambda KK, kk, Z, la, rh, X, ch=1 << 21:
                        good(KK, kk, Z, la, 0.0, X, ch))
    bad = OC.relative_residual(K, factors, kidx, oidx, vals, lam, rho, W, chunk=4)
    assert abs(bad - want) > 1e-3 * want


# ---------------------------------------------------- per-index Gram blocks
def test_segment_grams_are_the_blocks_of_FtF():
    """F'F = (I (x) K) H (I (x) K) with H block diagonal over kernel indices,
    block i = C_i (Appendix A.2 mixed-product rule); F from the literal
    selection-matrix form S'(Z (x) K).  K is positive definite here, so the
    blocks are recovered uniquely."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(n=5, q=23, r=3, seed=9,
                                                          other=(3, 4), sigma=0.3)
    n, r = K.shape[0], 3
    F = literal_F(K, factors, kidx, oidx)
    IKinv = np.kron(np.eye(r), np.linalg.inv(K))
    H = (IKinv @ (F.T @ F) @ IKinv).reshape(r, n, r, n)
    C = O.segment_grams(n, kidx, O.zhat(factors, oidx))
    for i in range(n):
        np.testing.assert_allclose(C[i], H[:, i, :, i], rtol=1e-8, atol=1e-8)
        for i2 in range(n):
            if i2 != i:
                assert np.abs(H[:, i, :, i2]).max() <= 1e-8
    # chunks of the observation list add up to the same blocks
    Zh = O.zhat(factors, oidx)
    C2 = O.segment_grams(n, kidx[:10], Zh[:10])
    O.segment_grams(n, kidx[10:], Zh[10:], C2)
    np.testing.assert_allclose(C2, C, rtol=1e-14, atol=1e-14)


def test_gram_form_of_the_product():
    """Yhat1(i,:) = C_i Xhat(i,:)' equals the gather-dot/scatter of Eqs. vl and
    yhat1, the Gram-form operator equals the dense literal system, and
    ||F vec(E)||^2 from the blocks equals the literal one."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(n=6, q=21, r=3, seed=10)
    n, r = K.shape[0], 3
    Zh = O.zhat(factors, oidx)
    C = O.segment_grams(n, kidx, Zh)
    X = np.random.default_rng(11).standard_normal((n, r))
    Xh = O.kernel_times(K, X)
    np.testing.assert_allclose(O.yhat1_from_grams(C, Xh),
                               O.scatter_rows(n, kidx, O.gather_dot(Xh, kidx, Zh), Zh),
                               rtol=1e-12, atol=1e-13)
    F = literal_F(K, factors, kidx, oidx)
    A = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    np.testing.assert_allclose(O.vec(O.matvec_grams(K, C, lam, rho, X)), A @ O.vec(X),
                               rtol=1e-12, atol=1e-12)
    fe = F @ O.vec(X)
    np.testing.assert_allclose(O.fitted_error_sq_grams(K, C, X), fe @ fe, rtol=1e-12)


# ----------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped term or a transposed operand planted in the oracle must make
    a pin fail (mistakes are planted in the oracle, on the CPU)."""
    K, factors, kidx, oidx, vals, lam, rho = tiny_problem(q=14, r=2)
    n, r = K.shape[0], 2
    F = literal_F(K, factors, kidx, oidx)
    A_lit = F.T @ F + lam * np.kron(np.eye(r), K) + rho * np.eye(n * r)
    X = np.random.default_rng(2).standard_normal((n, r))
    Zh = O.zhat(factors, oidx)
    good = O.vec(O.matvec(K, kidx, Zh, lam, rho, X))
    assert np.allclose(good, A_lit @ O.vec(X))
    # dropped lambda term
    bad = O.vec(O.matvec(K, kidx, Zh, 0.0, rho, X))
    assert not np.allclose(bad, A_lit @ O.vec(X), rtol=1e-6)
    # transposed kernel matrix on an unsymmetric perturbation
    Kp = K + 0.01 * np.triu(np.ones_like(K), 1)
    F2 = literal_F(Kp, factors, kidx, oidx)
    monkeypatch.setattr(OC, "kernel_times", lambda KK, XX: KK.T @ XX)
    bad2 = O.vec(OC.matvec(Kp, kidx, Zh, lam, rho, X))
    A2 = F2.T @ F2 + lam * np.kron(np.eye(r), Kp) + rho * np.eye(n * r)
    assert not np.allclose(bad2, A2 @ O.vec(X), rtol=1e-6)


def test_synthetic_sampling_is_uniform_without_replacement():
    rng = np.random.default_rng(0)
    kidx, oidx = synth.sample_observations(rng, 50, (7, 9), 2000)
    lin = kidx.astype(np.int64) * 63 + oidx[:, 0] + 7 * oidx[:, 1]
    assert len(np.unique(lin)) == 2000 and np.all(np.diff(lin) > 0)
    assert kidx.min() >= 0 and kidx.max() < 50 and oidx[:, 1].max() < 9
