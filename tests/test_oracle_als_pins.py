"""Pins of the alternating-fit oracle (oracle/als_oracle.py) to facts that do
not come from the oracle itself: a brute-force dense Kruskal tensor, the
optimality (zero gradient) of each finite-mode update, exact recovery of
planted noise-free factors, a planted mistake, and the monotone objective of
alternating minimisation (§2)."""
import numpy as np
import pytest

import oracle.als_oracle as A
import synth


def small(seed=0, n=12, other=(7, 9), q=500, r=3, noise=0.01):
    return synth.planted_problem(seed, n, other, q, r, bandwidth=0.2, lam=1e-3, rho=1e-6,
                                 noise=noise, shuffle=True)


def test_model_values_match_dense_kruskal_tensor():
    rng = np.random.default_rng(1)
    n, n1, n2, r = 5, 4, 6, 3
    K = synth.gaussian_kernel(synth.grid_points(n), 0.3)
    W = rng.standard_normal((n, r))
    F1, F2 = rng.standard_normal((n1, r)), rng.standard_normal((n2, r))
    Ak = K @ W
    T = np.zeros((n, n1, n2))
    for j in range(r):  # sum of outer products, written out
        for i in range(n):
            for a in range(n1):
                for b in range(n2):
                    T[i, a, b] += Ak[i, j] * F1[a, j] * F2[b, j]
    kidx = rng.integers(0, n, 40).astype(np.int32)
    oidx = np.stack([rng.integers(0, n1, 40), rng.integers(0, n2, 40)], 1).astype(np.int32)
    m = A.model_values(K, W, [F1, F2], kidx, oidx)
    np.testing.assert_allclose(m, T[kidx, oidx[:, 0], oidx[:, 1]], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1])
def test_finite_update_zeroes_the_gradient(mode):
    p = small(2, q=600)
    rng = np.random.default_rng(3)
    W = rng.standard_normal((p.n, p.r))
    new = A.finite_update(p.K, W, p.factors, mode, p.kidx, p.oidx, p.vals)
    facs = [np.array(F) for F in p.factors]
    facs[mode] = new
    counts = np.bincount(p.oidx[:, mode], minlength=new.shape[0])
    full = counts >= p.r  # rows without the ridge
    f = lambda F: A.objective(p.K, W, [F if k == mode else facs[k] for k in range(2)],
                              p.kidx, p.oidx, p.vals, p.lam, p.rho)
    eps = 1e-6
    scale = None
    for _ in range(4):
        E = rng.standard_normal(new.shape) * full[:, None]
        g = (f(new + eps * E) - f(new - eps * E)) / (2 * eps)
        # the same directional derivative at the old factor sets the scale
        g0 = (f(np.asarray(p.factors[mode]) + eps * E) - f(np.asarray(p.factors[mode]) - eps * E)) / (2 * eps)
        scale = max(scale or 0.0, abs(g0))
        assert abs(g) <= 1e-6 * max(scale, 1.0)


def test_finite_update_recovers_planted_factor():
    rng = np.random.default_rng(4)
    n, other, r, q = 10, (6, 8), 3, 480
    K = synth.gaussian_kernel(synth.grid_points(n), 0.2)
    W = rng.standard_normal((n, r))
    F = [rng.standard_normal((other[0], r)), rng.standard_normal((other[1], r))]
    kidx, oidx = synth.sample_observations(rng, n, other, q)
    t = A.model_values(K, W, F, kidx, oidx)  # noise-free
    start = [rng.standard_normal(F[0].shape), F[1]]
    got = A.finite_update(K, W, start, 0, kidx, oidx, t)
    counts = np.bincount(oidx[:, 0], minlength=other[0])
    assert np.all(counts >= r)
    np.testing.assert_allclose(got, F[0], rtol=1e-8, atol=1e-8)


def test_planted_mistake_is_caught(monkeypatch):
    # an update that forgets the kernel matrix (uses W for K W) cannot recover
    rng = np.random.default_rng(5)
    n, other, r, q = 10, (6, 8), 3, 480
    K = synth.gaussian_kernel(synth.grid_points(n), 0.2)
    W = rng.standard_normal((n, r))
    F = [rng.standard_normal((other[0], r)), rng.standard_normal((other[1], r))]
    kidx, oidx = synth.sample_observations(rng, n, other, q)
    t = A.model_values(K, W, F, kidx, oidx)
    monkeypatch.setattr(A, "kernel_factor", lambda K_, W_: np.asarray(W_))
    got = A.finite_update(K, W, [rng.standard_normal(F[0].shape), F[1]], 0, kidx, oidx, t)
    assert not np.allclose(got, F[0], rtol=1e-4, atol=1e-4)


def test_als_objective_never_increases():
    p = small(6, n=15, other=(8, 10), q=900, r=3, noise=0.05)
    rng = np.random.default_rng(7)
    facs = [rng.standard_normal(F.shape) for F in p.factors]
    W, facs, errs, objs = A.als(p.K, facs, p.kidx, p.oidx, p.vals, p.lam, p.rho, sweeps=4)
    for a, b in zip(objs, objs[1:]):
        assert b <= a * (1 + 1e-10) + 1e-12
    assert errs[-1] < errs[0]


def test_als_pcg_kernel_update_matches_direct():
    p = small(8, n=14, other=(6, 7), q=500, r=2)
    rng = np.random.default_rng(9)
    facs = [rng.standard_normal(F.shape) for F in p.factors]
    Wd, fd, ed, _ = A.als(p.K, facs, p.kidx, p.oidx, p.vals, p.lam, p.rho, sweeps=2)
    Wp, fp, ep, _ = A.als(p.K, facs, p.kidx, p.oidx, p.vals, p.lam, p.rho, sweeps=2,
                          method="pcg")
    np.testing.assert_allclose(ep, ed, rtol=1e-6)
