"""GPU parity: every step of the CUDA path against the FP64 CPU oracle, called
through the C ABI (via the ctypes binding).

Step outputs are compared element by element (tests/elementwise.py):
|a_ij - b_ij| <= tol (|b_ij| + max_k |b_ik|), one row per kernel index, so an
error confined to a short row (an index with one or two observations) cannot
hide under the long rows; rows of empty indices must be exactly zero.

Tolerances:
* index work (sort permutation, row pointer): bit-exact;
* FP64 steps (Zhat products, MTTKRP, gather-dot/scatter, Gram, operator,
  preconditioner): tol 1e-12 .. 1e-11 (sums of at most a few thousand terms;
  the eigenbasis round trip adds ~n eps);
* FP32 gather-dot/scatter and operator: the FP32 unit roundoff u32 = 6e-8
  times the growth of a sum of a few thousand terms;
* TF32 / BF16 tensor-core operators: the operand rounding (2^-11 and 2^-8
  per element) times the same growth;
* solves: the gate is the oracle's FP64 true relative residual
  ||b - A w|| / ||b|| <= tol and the relative error of the fitted values
  ||F(w - w*)|| / ||F w*|| <= 10 tol against the oracle's direct solution
  (the system's condition number, ~1e10 at lambda = 1e-4, rho = 1e-6, makes
  W itself sensitive); on well-conditioned cases W itself is gated.
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


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def make(ctx, pkg, p, sorted_obs=None, lowp=None):
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    if sorted_obs is None:
        sorted_obs = bool(np.all(np.diff(p.kidx) >= 0))
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r,
                       sorted_obs=sorted_obs, lowp=lowp)
    return kern, prob


CASES = {
    # name: (seed, n, other, q, r, shuffle)  -- several pieces per kernel index
    # (segments > 512 observations), ragged tails, empty kernel indices
    "long_segments": (1, 12, (40, 50), 14000, 5, True),
    "c1_shape": (0, 100, (20, 30), 6000, 5, False),
    "empty_rows": (2, 300, (3, 4), 500, 7, True),
    "three_modes_r16": (3, 64, (5, 6, 7), 9000, 16, True),
    "r1": (4, 30, (10,), 200, 1, True),
    "r64": (5, 50, (12, 14), 4000, 64, True),
    "r40": (6, 80, (30, 40), 30000, 40, False),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, ctx, pkg):
    seed, n, other, q, r, shuffle = CASES[request.param]
    p = synth.planted_problem(seed, n, other, q, r, bandwidth=0.1, lam=1e-4, rho=1e-6,
                              shuffle=shuffle)
    kern, prob = make(ctx, pkg, p)
    yield p, prob
    prob.close()
    kern.close()


def test_stable_sort_and_row_ptr_bit_exact(case):
    p, prob = case
    perm, rp = prob.order()
    np.testing.assert_array_equal(perm, np.argsort(p.kidx, kind="stable"))
    np.testing.assert_array_equal(rp, np.searchsorted(p.kidx[perm], np.arange(p.n + 1)))


def test_gram_and_eig(case):
    p, prob = case
    V, DV, UV = prob.gram()
    check_rows(V, O.gram(p.factors), 1e-13, "V")
    assert rel(V @ UV, UV * DV) <= 1e-12
    assert rel(UV.T @ UV, np.eye(p.r)) <= 1e-12


def test_rhs(case):
    p, prob = case
    B, b = prob.rhs()
    Zh = O.zhat(p.factors, p.oidx)
    Bo = O.mttkrp(p.n, p.kidx, p.vals, Zh)
    check_rows(B, Bo, 1e-12, "B")
    check_rows(b, p.K @ Bo, 1e-11, "K B")


# Element-wise bounds of the gather-dot/scatter per arithmetic.
GDS_TOL = {"fp64": 1e-12, "fp64_emulated": 1e-12, "mixed_fp32": 3e-5}


def test_gather_dot_scatter(case):
    p, prob = case
    Zh = O.zhat(p.factors, p.oidx)
    Xh = np.random.default_rng(11).standard_normal((p.n, p.r))
    ref = O.scatter_rows(p.n, p.kidx, O.gather_dot(Xh, p.kidx, Zh), Zh)
    for prec, tol in GDS_TOL.items():
        check_rows(prob.gds(Xh, prec), ref, tol, f"Yhat1 {prec}")


# Element-wise bounds of the operator (§4.4.1 product) per arithmetic.
MATVEC_TOL = {"fp64": 1e-11, "fp64_emulated": 1e-11, "mixed_fp32": 5e-5,
              "mixed_tf32": 1e-2, "mixed_bf16": 8e-2, "mixed_tf32x3": 5e-5,
              "mixed_bf16x3": 1e-4}


def test_matvec(case):
    p, prob = case
    Zh = O.zhat(p.factors, p.oidx)
    X = np.random.default_rng(12).standard_normal((p.n, p.r))
    for lam, rho in ((1e-4, 1e-6), (0.3, 0.05)):
        ref = O.matvec(p.K, p.kidx, Zh, lam, rho, X)
        for prec, tol in MATVEC_TOL.items():
            check_rows(prob.matvec(X, lam, rho, prec), ref, tol, f"A X {prec} lam={lam}")


@pytest.mark.parametrize("r", [8, 40, 64])
def test_fp64_accurate_products_several_chunks_and_splits(ctx, pkg, r):
    # n = 3000: 24 row tiles of 128 (the last one ragged) and the k range split
    # over several blocks, each more than one 256-wide exact chunk; a narrow
    # kernel (strongly graded D_K) makes the column scales of the products'
    # right-hand operand span many binades.  The FP64-accurate operator (both
    # n x n products and the gather/scatter) must stay at FP64 accuracy.
    p = synth.planted_problem(7, 3000, (20, 25), 20000, r, bandwidth=0.05, lam=1e-4, rho=1e-6,
                              shuffle=True)
    kern, prob = make(ctx, pkg, p)
    Zh = O.zhat(p.factors, p.oidx)
    X = np.random.default_rng(13).standard_normal((p.n, p.r))
    ref = O.matvec(p.K, p.kidx, Zh, 1e-4, 1e-6, X)
    check_rows(prob.matvec(X, 1e-4, 1e-6, "fp64"), ref, 1e-12, "A X fp64")
    check_rows(prob.matvec(X, 1e-4, 1e-6, "fp64_emulated"), ref, 1e-12, "A X fp64_emulated")
    prob.close()
    kern.close()


def test_tensor_core_products_at_n8000(ctx, pkg):
    # n = 8000 (the single-solve workload's kernel size): 63 row tiles of 128
    # with a ragged last one, the k range split over blocks, and every
    # tensor-core arithmetic of the operator, element by element.
    p = synth.planted_problem(14, 8000, (40, 50), 200000, 40, bandwidth=0.1, lam=1e-4,
                              rho=1e-6)
    kern, prob = make(ctx, pkg, p, sorted_obs=True)
    C = O.segment_grams(p.n, p.kidx, O.zhat(p.factors, p.oidx))
    X = np.random.default_rng(15).standard_normal((p.n, p.r))
    ref = O.matvec_grams(p.K, C, 1e-4, 1e-6, X)
    for prec, tol in MATVEC_TOL.items():
        check_rows(prob.matvec(X, 1e-4, 1e-6, prec), ref, tol, f"A X {prec} n=8000")
    prob.close()
    kern.close()


def test_preconditioner(case):
    p, prob = case
    X = np.random.default_rng(13).standard_normal((p.n, p.r))
    V = O.gram(p.factors)
    g = O.density(p.n, p.other_sizes, p.q)
    UK, UV, D = O.precond_setup(p.K, V, g, 0.3, 0.05)
    check_rows(prob.precond(X, 0.3, 0.05), O.precond_apply(UK, UV, D, X), 1e-10, "M^-1 X")


def _gate(p, W, tol, Wd=None):
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
    if Wd is None:
        Wd = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    Zh = O.zhat(p.factors, p.oidx)
    fit = rel(O.fitted_values(p.K, W, p.kidx, Zh), O.fitted_values(p.K, Wd, p.kidx, Zh))
    return res, fit, rel(W, Wd)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp64_emulated", 1e-10),
                                           ("mixed_fp32", 1e-6), ("mixed_fp32", 1e-8),
                                           ("mixed_fp32", 1e-10), ("mixed_tf32", 1e-6),
                                           ("mixed_tf32", 1e-8), ("mixed_bf16", 1e-6),
                                           ("mixed_bf16", 1e-8), ("mixed_tf32x3", 1e-6),
                                           ("mixed_tf32x3", 1e-10), ("mixed_bf16x3", 1e-6),
                                           ("mixed_bf16x3", 1e-10)])
def test_solve_c1_workload(ctx, pkg, precision, tol):
    """n=100, 20x30, q=6000, r=5, lambda=1e-4, rho=1e-6 (planted, 1% noise)."""
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=0)
    kern, prob = make(ctx, pkg, p, lowp=(precision != "fp64"))
    W, st = prob.solve(p.lam, p.rho, tol, max_iter=2000, precision=precision)
    res, fit, werr = _gate(p, W, tol)
    assert st["status"] == 0, st
    assert res <= tol, (res, st)
    assert fit <= 10 * tol, (fit, st)
    assert st["rel_residual"] <= tol
    prob.close()
    kern.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_solve_well_conditioned_W_itself(ctx, pkg, seed):
    p = synth.planted_problem(seed, 30, (8, 9), 1500, 6, bandwidth=0.08, lam=0.05, rho=1e-2,
                              shuffle=True)
    kern, prob = make(ctx, pkg, p)
    Wd = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    W, st = prob.solve(p.lam, p.rho, 1e-13, max_iter=500, precision="fp64")
    assert rel(W, Wd) <= 1e-10, st
    W2, st2 = prob.solve(p.lam, p.rho, 1e-10, max_iter=500, precision="mixed_fp32")
    assert rel(W2, Wd) <= 1e-8, st2
    W3, st3 = prob.solve(p.lam, p.rho, 1e-13, max_iter=500, precision="fp64_emulated")
    assert rel(W3, Wd) <= 1e-10, st3
    prob.close()
    kern.close()


def test_aligned_case_one_iteration(ctx, pkg):
    """Every entry observed: the preconditioner is the inverse (PCG: 1 step)."""
    p = synth.planted_problem(7, 20, (4, 5), 0, 3, bandwidth=0.15, lam=0.1, rho=1e-6,
                              aligned=True)
    kern, prob = make(ctx, pkg, p)
    W, st = prob.solve(p.lam, p.rho, 1e-10, max_iter=50, precision="fp64")
    assert st["iterations"] == 1, st
    res, fit, _ = _gate(p, W, 1e-10)
    assert res <= 1e-10
    prob.close()
    kern.close()


def test_unsorted_equals_sorted(ctx, pkg):
    p = synth.planted_problem(8, 60, (9, 11), 3000, 8, bandwidth=0.1, lam=1e-3, rho=1e-4)
    ps = synth.planted_problem(8, 60, (9, 11), 3000, 8, bandwidth=0.1, lam=1e-3, rho=1e-4)
    perm = np.random.default_rng(0).permutation(p.q)
    ps.kidx, ps.oidx, ps.vals = p.kidx[perm], p.oidx[perm], p.vals[perm]
    k1, pr1 = make(ctx, pkg, p, sorted_obs=True)
    k2, pr2 = make(ctx, pkg, ps, sorted_obs=False)
    W1, _ = pr1.solve(p.lam, p.rho, 1e-11, 1000)
    W2, _ = pr2.solve(p.lam, p.rho, 1e-11, 1000)
    assert rel(W1, W2) <= 1e-7
    for h in (pr1, pr2, k1, k2):
        h.close()


def test_fp32_values_equal_the_same_values_in_fp64(ctx, pkg):
    # CPHIFI_VALS_F32: float values are widened to FP64 on the device, exactly,
    # so the solve must give the same bits as the widened values passed as
    # doubles (host and device memory).
    import torch
    p = synth.planted_problem(16, 90, (12, 15), 5000, 6, bandwidth=0.1, lam=1e-4, rho=1e-6)
    v32 = p.vals.astype(np.float32)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    for prec in ("fp64", "mixed_fp32"):
        W64, s64 = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, v32.astype(np.float64), p.r,
                             p.lam, p.rho, 1e-9, 500, precision=prec, sorted_obs=True)
        W32, s32 = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, v32, p.r, p.lam, p.rho, 1e-9,
                             500, precision=prec, sorted_obs=True)
        np.testing.assert_array_equal(W32, W64)
        assert s32["iterations"] == s64["iterations"]
        dev = torch.device("cuda", 0)
        fac = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
        out = torch.empty(p.n * p.r, dtype=torch.float64, device=dev)
        pkg.solve(ctx, kern, fac, torch.from_numpy(p.kidx).to(dev),
                  torch.from_numpy(np.ascontiguousarray(p.oidx).ravel()).to(dev),
                  torch.from_numpy(v32).to(dev), p.r, p.lam, p.rho, 1e-9, 500, precision=prec,
                  sorted_obs=True, out=out)
        np.testing.assert_array_equal(out.cpu().numpy().reshape(p.r, p.n).T, W64)
    kern.close()


@pytest.mark.parametrize("vals32", [False, True])
def test_chunked_host_upload_equals_device_inputs(ctx, pkg, vals32):
    # Sorted host inputs with q >= 2^20 are uploaded in chunks that the Zhat
    # pass follows; the pass does the same arithmetic per piece, so the solve
    # must give the same bits as from device-resident inputs.
    import torch
    p = synth.planted_problem(17, 600, (60, 70), 1_500_000, 16, bandwidth=0.1, lam=1e-4,
                              rho=1e-6)
    vals = p.vals.astype(np.float32) if vals32 else p.vals
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    dev = torch.device("cuda", 0)
    fac = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
    outs = []
    for inputs in ("host", "device"):
        if inputs == "host":
            args = (p.factors, p.kidx, p.oidx, vals)
        else:
            args = (fac, torch.from_numpy(p.kidx).to(dev),
                    torch.from_numpy(np.ascontiguousarray(p.oidx).ravel()).to(dev),
                    torch.from_numpy(vals).to(dev))
        out = torch.empty(p.n * p.r, dtype=torch.float64, device=dev)
        W, st = pkg.solve(ctx, kern, *args, p.r, p.lam, p.rho, 1e-8, 500,
                          precision="mixed_fp32", sorted_obs=True, out=out)
        outs.append((out.cpu().numpy(), st["iterations"]))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    kern.close()


def test_deterministic(ctx, pkg):
    p = synth.planted_problem(9, 70, (15, 16), 8000, 12, bandwidth=0.1, lam=1e-4, rho=1e-6)
    kern, prob = make(ctx, pkg, p)
    for prec in ("fp64", "mixed_fp32", "fp64_emulated", "mixed_tf32", "mixed_bf16",
                 "mixed_tf32x3", "mixed_bf16x3"):
        W1, s1 = prob.solve(p.lam, p.rho, 1e-9, 500, precision=prec)
        W2, s2 = prob.solve(p.lam, p.rho, 1e-9, 500, precision=prec)
        np.testing.assert_array_equal(W1, W2)
        assert s1["iterations"] == s2["iterations"]
    prob.close()
    kern.close()


def test_warm_start(ctx, pkg):
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=1)
    kern, prob = make(ctx, pkg, p)
    W, st = prob.solve(p.lam, p.rho, 1e-10, 1000)
    W2, st2 = prob.solve(p.lam, p.rho, 1e-10, 1000, W0=W)
    assert st2["iterations"] <= 2, st2
    assert O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W2) <= 1e-10
    prob.close()
    kern.close()


def test_empty_observations(ctx, pkg):
    p = synth.planted_problem(10, 16, (3, 4), 0, 3)
    kern, prob = make(ctx, pkg, p)
    W, st = prob.solve(p.lam, p.rho, 1e-10, 100)
    assert st["status"] == 0 and np.all(W == 0)
    prob.close()
    kern.close()


def test_not_converged_reports(ctx, pkg):
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=2)
    kern, prob = make(ctx, pkg, p)
    W, st = prob.solve(p.lam, p.rho, 1e-14, max_iter=3, raise_on_error=False)
    assert st["status"] == pkg.E_NOT_CONVERGED and st["iterations"] == 3
    assert np.all(np.isfinite(W)) and st["rel_residual"] > 1e-14
    prob.close()
    kern.close()


def test_invalid_inputs_are_rejected(ctx, pkg):
    p = synth.planted_problem(11, 20, (4, 5), 100, 3)
    dK, UK = np.linalg.eigh(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    bad = p.kidx.copy()
    bad[17] = p.n
    with pytest.raises(pkg.CphifiError) as e:
        pkg.Problem(ctx, kern, p.factors, bad, p.oidx, p.vals, p.r)
    assert e.value.status == pkg.E_INVALID_ARG
    badv = p.vals.copy()
    badv[3] = np.nan
    with pytest.raises(pkg.CphifiError):
        pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, badv, p.r)
    bado = p.oidx.copy()
    bado[5, 1] = -1
    with pytest.raises(pkg.CphifiError):
        pkg.Problem(ctx, kern, p.factors, p.kidx, bado, p.vals, p.r)
    shuffled = p.kidx[::-1].copy()
    with pytest.raises(pkg.CphifiError):
        pkg.Problem(ctx, kern, p.factors, shuffled, p.oidx[::-1].copy(), p.vals[::-1].copy(),
                    p.r, sorted_obs=True)
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r)
    with pytest.raises(pkg.CphifiError):
        prob.solve(p.lam, 0.0, 1e-8)
    prob.close()
    kern.close()


def test_admission_by_budget(pkg):
    p = synth.planted_problem(12, 40, (10, 10), 2000, 4)
    dK, UK = np.linalg.eigh(p.K)
    # room for the kernel handle (U_K in FP64 + hi/lo FP32, D_K) but not the problem
    c = pkg.Context(0, hbm_budget_bytes=40 * 40 * 16 + 40 * 8 + 4096)
    kern = c.kernel_create(p.n, UK, dK)
    with pytest.raises(pkg.CphifiError) as e:
        pkg.Problem(c, kern, p.factors, p.kidx, p.oidx, p.vals, p.r)
    assert e.value.status == pkg.E_ADMISSION
    kern.close()
    c.close()


def test_device_pointers(ctx, pkg):
    import torch
    p = synth.planted_problem(13, 50, (10, 12), 3000, 5, lam=1e-3, rho=1e-5)
    dK, UK = np.linalg.eigh(p.K)
    kern = ctx.kernel_create(p.n, torch.from_numpy(np.asfortranarray(UK).ravel(order="F")).cuda(),
                             torch.from_numpy(dK).cuda())
    fac = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).cuda() for F in p.factors]
    out = torch.empty(p.n * p.r, dtype=torch.float64, device="cuda")
    W, st = pkg.solve(ctx, kern, fac, torch.from_numpy(p.kidx).cuda(),
                      torch.from_numpy(p.oidx.ravel()).cuda(), torch.from_numpy(p.vals).cuda(),
                      p.r, p.lam, p.rho, 1e-10, 1000, out=out, sorted_obs=True)
    Wh = out.cpu().numpy().reshape(p.r, p.n).T
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, Wh)
    assert st["status"] == 0 and res <= 1e-10
    kern.close()


# Slowly converging instances of the uneven batch: Matern-3/2 kernels with few
# observations per unknown (q ~ 1e3 for n r ~ 3e3 .. 3e4), where FP64 PCG
# needs hundreds of iterations and the preconditioner's density weight gamma
# is small.  The mixed modes must still reach the tolerance on the oracle's
# FP64 true residual, restarting only when the low-precision recurrence
# drifts.
HARD = {
    "matern_n105_q1040_r32": dict(n=105, other_sizes=(58, 58), q=1040, r=32, kernel="matern32",
                                  seed=845932451),
    "matern_n1223_q1107_r32": dict(n=1223, other_sizes=(61, 60), q=1107, r=32,
                                   kernel="matern32", seed=546953866),
    "matern_n457_q2429_r32": dict(n=457, other_sizes=(62, 62), q=2429, r=32, kernel="matern32",
                                  seed=1745629169),
}


@pytest.mark.parametrize("name", list(HARD))
@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_tf32x3", "mixed_bf16x3", "fp64_emulated"])
def test_slow_instances_reach_tolerance(ctx, pkg, name, prec):
    p = synth.batch_problem(HARD[name])
    dK, UK = np.linalg.eigh(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    W, st = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-6,
                      max_iter=6000, precision=prec, sorted_obs=True)
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
    assert st["status"] == 0, st
    assert res <= 1e-6, (res, st)
    kern.close()


def test_kernel_from_K_with_device_eigensolver(ctx, pkg):
    # eig(K) computed on the device (Eq. eigK) gives the same solve as the
    # host eigendecomposition: the oracle's FP64 residual meets the tolerance
    # and the fitted values agree (W is invariant to the eigenvector basis).
    p = synth.planted_problem(21, 120, (20, 30), 6000, 5, bandwidth=0.1, lam=1e-4, rho=1e-6)
    kd = ctx.kernel_create(p.n, None, None, K=p.K)
    dK, UK = np.linalg.eigh(p.K)
    kh = ctx.kernel_create(p.n, UK, dK)
    Wd, sd = pkg.solve(ctx, kd, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-10,
                       2000, sorted_obs=True)
    Wh, sh = pkg.solve(ctx, kh, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-10,
                       2000, sorted_obs=True)
    assert sd["status"] == 0
    assert O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, Wd) <= 1e-10
    Zh = O.zhat(p.factors, p.oidx)
    fd, fh = O.fitted_values(p.K, Wd, p.kidx, Zh), O.fitted_values(p.K, Wh, p.kidx, Zh)
    assert rel(fd, fh) <= 1e-9
    bad = p.K.copy()
    bad[3, 4] = np.nan
    with pytest.raises(pkg.CphifiError) as e:
        ctx.kernel_create(p.n, None, None, K=bad)
    assert e.value.status == pkg.E_INVALID_ARG
    kd.close()
    kh.close()
