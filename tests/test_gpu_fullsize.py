"""Parity at the benchmark's full size (n = 8000, 400 x 500, q = 5e7, r = 40,
FP32 observation values), in the launch configuration bench.py times
(device-resident sorted inputs).

At this size the oracle cannot assemble the system, but it can hold the
per-index Gram blocks C_i = sum over l with i_l = i of Zhat(l,:)'Zhat(l,:)
(n r^2 values: the diagonal blocks of H in F'F = (I (x) K) H (I (x) K),
pinned against the literal F on tiny inputs), formed from the oracle's own
Zhat (Eq. zhat) by chunks of observations.  With them:

* every row of the gather-dot/scatter (Eqs. vl, yhat1) is checked element by
  element: Yhat1(i,:) = C_i Xhat(i,:)';
* the FP64 true relative residual ||K B - A vec(W)|| / ||K B|| of each
  returned W must meet the tolerance the solve was given;
* the oracle's own FP64 PCG (Gram-form operator, Eq. fx preconditioner)
  gives the reference W*, and the fitted values' relative error
  ||F(w - w*)|| / ||F w*|| (from the blocks) must be <= 10 tol;

for the mixed FP32 operator at 1e-6 and 1e-8 and the TF32, BF16 and 3-term
split-TF32 tensor-core operators at 1e-6.
"""
import numpy as np
import pytest

import oracle as O
import synth
from elementwise import check_rows
from kcache import eigh_cached

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(2400)]


@pytest.fixture(scope="module")
def full():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as pkg

    p = synth.workload("c3_mixed_n8000_q5e7_r40", seed=0)
    vals32 = p.vals.astype(np.float32)     # the workload's values are FP32
    p.vals = vals32.astype(np.float64)     # ... and the oracle sees exactly those
    n, r, q = p.n, p.r, p.q
    dK, UK = eigh_cached(p.K)
    ctx = pkg.Context(0)
    kern = ctx.kernel_create(n, UK, dK)
    dev = torch.device("cuda", 0)
    kd = torch.from_numpy(p.kidx).to(dev)
    od = torch.from_numpy(np.ascontiguousarray(p.oidx).ravel()).to(dev)
    vd = torch.from_numpy(vals32).to(dev)
    fd = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
    prob = pkg.Problem(ctx, kern, fd, kd, od, vd, r, sorted_obs=True, lowp=True)

    # the oracle: Gram blocks and the MTTKRP by chunks of observations
    C = np.zeros((n, r, r))
    B = np.zeros((n, r))
    chunk = 1 << 21
    for s in range(0, q, chunk):
        e = min(q, s + chunk)
        Zc = O.zhat(p.factors, p.oidx[s:e])
        O.segment_grams(n, p.kidx[s:e], Zc, C)
        B += O.mttkrp(n, p.kidx[s:e], p.vals[s:e], Zc)
    b = p.K @ B
    V = O.gram(p.factors)
    UKo, UV, D = O.precond_setup(p.K, V, O.density(n, p.other_sizes, q), p.lam, p.rho,
                                 eigK=(dK, UK))
    Ws, its, hist = O.pcg(lambda X: O.matvec_grams(p.K, C, p.lam, p.rho, X), b,
                          lambda R: O.precond_apply(UKo, UV, D, R), tol=1e-11, maxit=300)
    assert hist[-1] <= 1e-11, (its, hist[-1])
    yield dict(pkg=pkg, p=p, prob=prob, C=C, b=b, Ws=Ws,
               fw=np.sqrt(O.fitted_error_sq_grams(p.K, C, Ws)))
    prob.close()
    kern.close()
    ctx.close()


def test_full_size_gather_dot_scatter_every_row(full):
    p, prob, C = full["p"], full["prob"], full["C"]
    Xh = np.random.default_rng(3).standard_normal((p.n, p.r))
    ref = O.yhat1_from_grams(C, Xh)
    check_rows(prob.gds(Xh, "fp64_emulated"), ref, 1e-12, "Yhat1 double-float, n=8000 q=5e7")
    check_rows(prob.gds(Xh, "mixed_fp32"), ref, 1e-4, "Yhat1 FP32, n=8000 q=5e7")


@pytest.mark.parametrize("precision,tol", [("mixed_fp32", 1e-6), ("mixed_fp32", 1e-8),
                                           ("mixed_tf32", 1e-6), ("mixed_bf16", 1e-6),
                                           ("mixed_tf32x3", 1e-6), ("mixed_bf16x3", 1e-6),
                                           ("mixed_bf16x3", 1e-8)])
def test_full_size_solve(full, precision, tol):
    p, prob, C, b, Ws = full["p"], full["prob"], full["C"], full["b"], full["Ws"]
    W, st = prob.solve(p.lam, p.rho, tol, 500, precision=precision)
    assert st["status"] == full["pkg"].OK, st
    R = b - O.matvec_grams(p.K, C, p.lam, p.rho, W)
    res = np.linalg.norm(R) / np.linalg.norm(b)
    assert res <= tol, (res, st)
    # the library's own FP64-accurate residual agrees with the oracle's
    assert abs(st["rel_residual"] - res) <= 0.05 * res, (st["rel_residual"], res)
    fit = np.sqrt(O.fitted_error_sq_grams(p.K, C, W - Ws)) / full["fw"]
    assert fit <= 10 * tol, (fit, st)
