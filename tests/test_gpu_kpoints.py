"""Kernel matrices from design points (§2: K(i, j) = k(x_i, x_j) on the kernel
mode's points), through the C ABI, against the oracle and NumPy:

* cphifi_kernel_create_points builds K on the device and decomposes it
  (Eq. eigK): U_K diag(D_K) U_K' equals the K that the synthetic-input module
  draws for the same points, entry by entry (1e-12 of max |K|), and D_K
  equals NumPy's eigenvalues of that K (1e-12 of ||K||_2);
* cphifi_kernel_apply, Y = K X with K's tiles generated on the fly, against
  K @ X element by element: FP64 within 1e-12, FP32 (hardware exponential)
  within 2e-5; without points, the FP64 eigen form within 1e-11;
* the alternating fit with a points kernel (A_k = K W from the points)
  matches the oracle's loop as the stored-K fit does.
"""
import numpy as np
import pytest

import oracle.als_oracle as A
import synth
from elementwise import check_rows
from kcache import eigh_cached

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _euclid_kernel(P, kind, s):
    d = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    if kind == "gaussian":
        return np.exp(-(d * d) / (2 * s * s))
    u = np.sqrt(3.0) * d / s
    return (1 + u) * np.exp(-u)


# n = 1500: the column range of K split over 10 blocks per row block (the
# last split shorter), partial products added in split order
@pytest.mark.parametrize("kind,n,dim,s", [("gaussian", 300, 1, 0.1), ("matern32", 257, 1, 0.1),
                                          ("gaussian", 200, 2, 0.3), ("matern32", 1, 1, 0.5),
                                          ("matern32", 1500, 1, 0.1)])
def test_kernel_from_points(ctx, pkg, kind, n, dim, s):
    if dim == 1:
        x = synth.grid_points(n)
        K = synth.gaussian_kernel(x, s) if kind == "gaussian" else synth.matern32_kernel(x, s)
        P = x[:, None]
    else:
        P = np.random.default_rng(n).uniform(size=(n, dim))
        K = _euclid_kernel(P, kind, s)
    kern = ctx.kernel_from_points(P, kind, s)
    d, U = kern.eig()
    kmax = np.abs(K).max()
    assert np.abs((U * d) @ U.T - K).max() <= 1e-12 * kmax
    dref = np.linalg.eigvalsh(K)
    assert np.abs(d - dref).max() <= 1e-12 * np.abs(dref).max()
    X = np.random.default_rng(7).standard_normal((n, 24))
    check_rows(kern.apply(X, "fp64"), K @ X, 1e-12, "K X from points, FP64")
    check_rows(kern.apply(X, "mixed_fp32"), K @ X, 2e-5, "K X from points, FP32")
    kern.close()


def test_apply_without_points_uses_the_eigen_form(ctx, pkg):
    x = synth.grid_points(150)
    K = synth.gaussian_kernel(x, 0.1)
    dK, UK = eigh_cached(K)
    kern = ctx.kernel_create(150, UK, dK)
    X = np.random.default_rng(8).standard_normal((150, 7))
    check_rows(kern.apply(X, "fp64"), K @ X, 1e-11, "K X eigen form")
    kern.close()


def test_bad_points_rejected(ctx, pkg):
    with pytest.raises(pkg.CphifiError):
        ctx.kernel_from_points(np.array([0.0, np.nan, 1.0]), "gaussian", 0.1)
    with pytest.raises(pkg.CphifiError):
        ctx.kernel_from_points(np.linspace(0, 1, 5), "gaussian", 0.0)
    with pytest.raises(pkg.CphifiError) as e:
        ctx.kernel_from_points(np.linspace(0, 1, 4097), "gaussian", 0.1)
    assert e.value.status == pkg.E_UNSUPPORTED


def test_als_with_points_kernel_matches_oracle(ctx, pkg):
    p = synth.planted_problem(1, 40, (20, 25), 6000, 6, bandwidth=0.15, lam=1e-2, rho=1e-3,
                              shuffle=True)
    rng = np.random.default_rng(14)
    start = [rng.standard_normal(F.shape) for F in p.factors]
    Wo, fo, eo, _ = A.als(p.K, start, p.kidx, p.oidx, p.vals, p.lam, p.rho, sweeps=4)
    kern = ctx.kernel_from_points(synth.grid_points(p.n), "gaussian", 0.15)
    Wg, fg, eg, st = pkg.als(ctx, kern, start, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho,
                             tol=1e-12, sweeps=4, max_iter=5000, precision="fp64")
    np.testing.assert_allclose(eg, eo, rtol=1e-7)
    assert np.linalg.norm(Wg - Wo) <= 1e-5 * np.linalg.norm(Wo)
    kern.close()
