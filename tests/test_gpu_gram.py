"""The compressed-Gram form of the matrix-free product (§4.4.1, Eqs. vl and
yhat1 with the sum over each kernel index's observations done once):
C_i = sum over l with i_l = i of Zhat(l,:)'Zhat(l,:), Yhat1(i,:) = C_i
Xhat(i,:)'.  Checked through the C ABI against the oracle's segment_grams
(pinned against the literal F'F on tiny inputs), element by element:

* the blocks themselves (cphifi_problem_grams): FP64-accurate ones from the
  FP32 pair and from the FP64 copy of Zhat, tol 1e-12; FP32 ones (sums of up
  to ~1e4 FP32 products per element, accumulated per 32-observation tile),
  tol 5e-5;
* the product through the blocks (CPHIFI_GRAM_FORM) against the oracle's
  streamed form, with the bounds of the streamed product;
* solves with gram = 1 (iterations through the blocks) and gram = 2 (checks
  too), gated like the streamed solves: the oracle's FP64 true residual <= tol
  and the fitted values within 10 tol of the direct solution;
* new factors (the alternating fit) rebuild the blocks.
"""
import numpy as np
import pytest

import oracle as O
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


CASES = {
    # (seed, n, other, q, r, shuffle): several pieces per index, many pieces
    # per index, empty indices and a ragged tail, r = 1, 16 (three modes), 40, 64
    "long_segments": (1, 12, (40, 50), 14000, 5, True),
    "few_indices": (22, 4, (100, 60), 20000, 40, False),
    "empty_rows": (2, 300, (3, 4), 500, 7, True),
    "three_modes_r16": (3, 64, (5, 6, 7), 9000, 16, True),
    "r1": (4, 30, (10,), 200, 1, True),
    "r64": (5, 50, (12, 14), 4000, 64, True),
}


def _flat(C):
    n, r, _ = C.shape
    return C.reshape(n * r, r)   # one row per (index, j): element-wise with row maxima


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("lowp", [True, False])
def test_gram_blocks_and_products(ctx, pkg, name, lowp):
    seed, n, other, q, r, shuffle = CASES[name]
    p = synth.planted_problem(seed, n, other, q, r, bandwidth=0.1, lam=1e-4, rho=1e-6,
                              shuffle=shuffle)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, lowp=lowp)
    Zh = O.zhat(p.factors, p.oidx)
    Cref = O.segment_grams(p.n, p.kidx, Zh)
    wide = "fp64_emulated" if lowp else "fp64"
    check_rows(_flat(prob.grams(wide)), _flat(Cref), 1e-12, f"C_i {wide}")
    check_rows(_flat(prob.grams("mixed_fp32")), _flat(Cref), 5e-5, "C_i FP32")
    Xh = np.random.default_rng(11).standard_normal((p.n, p.r))
    ref = O.scatter_rows(p.n, p.kidx, O.gather_dot(Xh, p.kidx, Zh), Zh)
    check_rows(prob.gds(Xh, wide + "+gram"), ref, 1e-12, "Yhat1 from FP64-accurate blocks")
    check_rows(prob.gds(Xh, "mixed_fp32+gram"), ref, 5e-5, "Yhat1 from FP32 blocks")
    X = np.random.default_rng(12).standard_normal((p.n, p.r))
    mref = O.matvec(p.K, p.kidx, Zh, 1e-4, 1e-6, X)
    check_rows(prob.matvec(X, 1e-4, 1e-6, wide + "+gram"), mref, 1e-11, "A X Gram FP64")
    check_rows(prob.matvec(X, 1e-4, 1e-6, "mixed_fp32+gram"), mref, 5e-5, "A X Gram FP32")
    prob.close()
    kern.close()


def _gate(p, W, tol, Wd):
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
    Zh = O.zhat(p.factors, p.oidx)
    fw = O.fitted_values(p.K, Wd, p.kidx, Zh)
    fit = np.linalg.norm(O.fitted_values(p.K, W, p.kidx, Zh) - fw) / np.linalg.norm(fw)
    return res, fit


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp64_emulated", 1e-10),
                                           ("mixed_fp32", 1e-6), ("mixed_fp32", 1e-10),
                                           ("mixed_tf32", 1e-8), ("mixed_tf32x3", 1e-8),
                                           ("mixed_bf16x3", 1e-8)])
@pytest.mark.parametrize("gram", [1, 2])
def test_gram_solves_c1_workload(ctx, pkg, precision, tol, gram):
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=0)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, sorted_obs=True)
    W, st = prob.solve(p.lam, p.rho, tol, max_iter=2000, precision=precision, gram=gram)
    Wd = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    res, fit = _gate(p, W, tol, Wd)
    assert st["status"] == 0, st
    assert res <= tol, (res, st)
    assert fit <= 10 * tol, (fit, st)
    prob.close()
    kern.close()


def test_gram_blocks_follow_new_factors(ctx, pkg):
    p = synth.planted_problem(17, 40, (9, 11), 2500, 6, bandwidth=0.1)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, sorted_obs=True,
                       keep_obs=True)
    prob.grams("fp64_emulated")
    rng = np.random.default_rng(18)
    new = [rng.standard_normal(F.shape) for F in p.factors]
    prob.set_factors(new)
    Cref = O.segment_grams(p.n, p.kidx, O.zhat(new, p.oidx))
    check_rows(_flat(prob.grams("fp64_emulated")), _flat(Cref), 1e-12, "C_i after new factors")
    check_rows(_flat(prob.grams("mixed_fp32")), _flat(Cref), 5e-5, "C_i FP32 after new factors")
    prob.close()
    kern.close()
