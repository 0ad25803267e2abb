"""The device eigendecomposition of the kernel matrix (Eq. eigK, §3.2),
computed by the library's own Jacobi kernels when only K is passed to
cphifi_kernel_create, read back with cphifi_kernel_eig and checked against
NumPy's FP64 eigh:

* eigenvalues element by element: |d_k - d*_k| <= 1e-12 ||K||_2 (both
  ascending; eigenvalues are unique, eigenvectors are not);
* every eigenpair: ||K u_k - d_k u_k|| <= 1e-12 ||K||_2;
* orthogonality element by element: |(U'U - I)_jk| <= 1e-12 (about n eps
  for the rotations accumulated over all sweeps);

on Gaussian and Matern kernels (PSD, eigenvalues spread over 16 decades and
clustered near zero), odd and even n (the padded round-robin schedule), a
symmetric indefinite matrix, and the degenerate n = 1 and n = 2.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def _matrix(kind, n, seed):
    x = synth.grid_points(n)
    if kind == "gaussian":
        return synth.gaussian_kernel(x, 0.1)
    if kind == "matern":
        return synth.matern32_kernel(x, 0.1)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A + A.T


@pytest.mark.parametrize("kind,n", [("gaussian", 1), ("gaussian", 2), ("gaussian", 37),
                                    ("matern", 128), ("gaussian", 700), ("indefinite", 301),
                                    ("matern", 2000)])
def test_device_eig_against_numpy(ctx, kind, n):
    K = _matrix(kind, n, n)
    kern = ctx.kernel_create(n, None, None, K=K)
    d, U = kern.eig()
    kern.close()
    dref = np.linalg.eigvalsh(K)
    knorm = max(abs(dref[0]), abs(dref[-1]))
    assert np.all(np.diff(d) >= 0)
    np.testing.assert_array_less(np.abs(d - dref), 1e-12 * knorm + 1e-300)
    res = np.linalg.norm(K @ U - U * d, axis=0)
    assert res.max() <= 1e-12 * knorm, res.max() / knorm
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12


def test_device_eig_rejects_large_n_and_bad_values(ctx):
    import paper_2603_25691_gb300 as pkg
    with pytest.raises(pkg.CphifiError) as e:
        ctx.kernel_create(4097, None, None, K=np.eye(4097))
    assert e.value.status == pkg.E_UNSUPPORTED
    K = _matrix("gaussian", 20, 0)
    K[3, 1] = np.inf
    with pytest.raises(pkg.CphifiError) as e:
        ctx.kernel_create(20, None, None, K=K)
    assert e.value.status == pkg.E_INVALID_ARG
