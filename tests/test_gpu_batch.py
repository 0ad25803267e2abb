"""Batches of independent solves through cphifi_submit / cphifi_poll /
cphifi_wait, against the one-shot cphifi_solve and the FP64 oracle.

Each ALS sweep of CP-HIFI solves one independent kernel-mode subproblem
(§4.4) per tensor and mode; a batch runs many of them concurrently, each on a
stream of its own with its PCG chunks replayed from CUDA graphs.  Every kernel
of the path is deterministic (no floating-point atomics; launch shapes depend
only on the problem and the GPU), so a solve gives the same bits alone and in
a batch: W is compared bit for bit with the one-shot call, and one solve per
batch is also gated by the oracle's FP64 true residual.
"""
import numpy as np
import pytest

import oracle as O
import synth
from kcache import eigh_cached

# every test here drives host-side request loops: bound each one
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as p
    return p


# (seed, n, other sizes, q, r, precision, tol)
MIX = [
    (31, 100, (20, 30), 6000, 5, "fp64", 1e-10),
    (32, 300, (30, 40), 40000, 16, "mixed_fp32", 1e-8),
    (33, 64, (5, 6, 7), 9000, 16, "mixed_tf32x3", 1e-8),
    (34, 120, (25, 25), 20000, 40, "fp64_emulated", 1e-10),
    (35, 50, (12, 14), 4000, 64, "mixed_bf16", 1e-6),
    (36, 200, (50, 60), 30000, 24, "mixed_tf32", 1e-6),
    (37, 30, (10,), 200, 1, "mixed_fp32", 1e-8),
    (38, 300, (3, 4), 500, 7, "fp64", 1e-10),
]


def _problems():
    out = []
    for seed, n, other, q, r, prec, tol in MIX:
        p = synth.planted_problem(seed, n, other, q, r, bandwidth=0.1, lam=1e-4, rho=1e-6,
                                  shuffle=True)
        out.append((p, prec, tol))
    return out


@pytest.fixture(scope="module")
def batch(pkg):
    ctx = pkg.Context(0)
    probs = _problems()
    kerns = []
    for p, _, _ in probs:
        dK, UK = np.linalg.eigh(p.K)
        kerns.append(ctx.kernel_create(p.n, UK, dK))
    alone = []
    for (p, prec, tol), k in zip(probs, kerns):
        alone.append(pkg.solve(ctx, k, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho,
                               tol, max_iter=2000, precision=prec))
    yield ctx, probs, kerns, alone
    for k in kerns:
        k.close()
    ctx.close()


def _submit_all(pkg, ctx, probs, kerns):
    return [pkg.submit(ctx, k, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                       max_iter=2000, precision=prec)
            for (p, prec, tol), k in zip(probs, kerns)]


def test_batch_results_equal_alone(pkg, batch):
    ctx, probs, kerns, alone = batch
    reqs = _submit_all(pkg, ctx, probs, kerns)
    # wait in reverse order: completion order must not matter
    res = [None] * len(reqs)
    for i in reversed(range(len(reqs))):
        res[i] = reqs[i].wait()
    for (W, st), (Wa, sta), (p, prec, tol) in zip(res, alone, probs):
        assert st["status"] == pkg.OK, (prec, st)
        assert st["iterations"] == sta["iterations"]
        assert st["true_residuals"] == sta["true_residuals"]
        np.testing.assert_array_equal(W, Wa)
    # and the oracle's FP64 residual gates each result
    for (W, st), (p, prec, tol) in zip(res, probs):
        res_ = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
        assert res_ <= tol, (prec, res_)


def test_batch_repeat_replays_graphs(pkg, batch):
    ctx, probs, kerns, alone = batch
    for _ in range(2):
        reqs = _submit_all(pkg, ctx, probs, kerns)
        for r_, (Wa, _) in zip(reqs, alone):
            W, st = r_.wait()
            np.testing.assert_array_equal(W, Wa)


def test_slots_queue_requests(pkg, batch):
    ctx, probs, kerns, alone = batch
    ctx.set_slots(2)
    try:
        reqs = _submit_all(pkg, ctx, probs, kerns)
        active, pending = ctx.poll()
        assert active <= 2 and active + pending <= len(reqs)
        assert pending >= len(reqs) - 2 - 1  # at most one finished already
        for r_, (Wa, _) in zip(reqs, alone):
            W, _ = r_.wait()
            np.testing.assert_array_equal(W, Wa)
        assert ctx.poll() == (0, 0)
    finally:
        ctx.set_slots(16)


def test_budget_admission(pkg):
    # Under a small HBM budget, requests beyond what fits wait for memory to
    # free up and still give the same bits; a request that cannot fit even
    # alone completes with E_ADMISSION.
    probs = _problems()[:3]
    ctx0 = pkg.Context(0)
    p, prec, tol = probs[1]
    dK, UK = np.linalg.eigh(p.K)
    k = ctx0.kernel_create(p.n, UK, dK)
    ref, _ = pkg.solve(ctx0, k, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                       max_iter=2000, precision=prec)
    k.close()
    ctx0.close()

    budget = 64 << 20
    ctx = pkg.Context(0, hbm_budget_bytes=budget)
    try:
        dK, UK = np.linalg.eigh(p.K)
        k = ctx.kernel_create(p.n, UK, dK)
        reqs = [pkg.submit(ctx, k, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                           max_iter=2000, precision=prec) for _ in range(4)]
        for r_ in reqs:
            W, st = r_.wait()
            np.testing.assert_array_equal(W, ref)
        big = synth.planted_problem(40, 300, (200, 200), 2_000_000, 32, bandwidth=0.1)
        dK, UK = eigh_cached(big.K)
        kb = ctx.kernel_create(big.n, UK, dK)
        rq = pkg.submit(ctx, kb, big.factors, big.kidx, big.oidx, big.vals, big.r, 1e-4, 1e-6,
                        1e-8, precision="mixed_fp32")
        with pytest.raises(pkg.CphifiError) as e:
            rq.wait()
        assert e.value.status == pkg.E_ADMISSION
        kb.close()
        k.close()
    finally:
        ctx.close()


def test_wait_timeout_leaves_request_running(pkg, batch):
    ctx, probs, kerns, alone = batch
    p, prec, tol = probs[3]
    rq = pkg.submit(ctx, kerns[3], p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                    max_iter=2000, precision=prec)
    with pytest.raises(pkg.CphifiError) as e:
        rq.wait(timeout_us=0)
    assert e.value.status == pkg.E_TIMEOUT
    W, st = rq.wait()
    np.testing.assert_array_equal(W, alone[3][0])


def test_device_inputs_and_outputs(pkg, batch):
    import torch
    ctx, probs, kerns, alone = batch
    dev = torch.device("cuda", 0)
    reqs = []
    for (p, prec, tol), k in list(zip(probs, kerns))[:4]:
        f = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
        ki = torch.from_numpy(p.kidx.astype(np.int32)).to(dev)
        oi = torch.from_numpy(np.ascontiguousarray(p.oidx, dtype=np.int32)).to(dev)
        v = torch.from_numpy(p.vals).to(dev)
        reqs.append(pkg.submit(ctx, k, f, ki, oi, v, p.r, p.lam, p.rho, tol, max_iter=2000,
                               precision=prec))
    for r_, (p, prec, tol), (Wa, _) in zip(reqs, probs, alone):
        W, st = r_.wait()
        W = W.cpu().numpy().reshape(p.r, p.n).T
        np.testing.assert_array_equal(W, Wa)


def test_submit_rejects_bad_arguments(pkg, batch):
    ctx, probs, kerns, alone = batch
    p, prec, tol = probs[0]
    with pytest.raises(pkg.CphifiError) as e:
        pkg.submit(ctx, kerns[0], p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, -1.0, tol)
    assert e.value.status == pkg.E_INVALID_ARG
    with pytest.raises(pkg.CphifiError) as e:
        ctx.set_slots(0)
    assert e.value.status == pkg.E_INVALID_ARG


def test_poll_lists_completed_tickets(pkg, batch):
    ctx, probs, kerns, alone = batch
    reqs = _submit_all(pkg, ctx, probs, kerns)
    want = {r_.ticket for r_ in reqs}
    seen = []
    for _ in range(2_000_000):
        active, pending, done = ctx.poll(done_cap=3)
        seen += done
        if active == 0 and pending == 0 and len(seen) == len(want):
            break
    assert sorted(seen) == sorted(want) and len(set(seen)) == len(seen)
    for r_, (Wa, _) in zip(reqs, alone):
        W, st = r_.wait(timeout_us=0)  # already complete: returns at once
        np.testing.assert_array_equal(W, Wa)
    assert ctx.poll(done_cap=8) == (0, 0, [])


def test_invalid_inputs_fail_the_request_only(pkg, batch):
    # A submitted problem is created without waiting on the device; its input
    # errors surface when the request completes, and the requests around it
    # are unaffected.
    ctx, probs, kerns, alone = batch
    p, prec, tol = probs[0]
    bad_k = p.kidx.copy()
    bad_k[len(bad_k) // 2] = p.n + 3
    order = np.argsort(p.kidx, kind="stable")
    unsorted_k = p.kidx[order][::-1].copy()
    unsorted_o = p.oidx[order][::-1].copy()
    unsorted_v = p.vals[order][::-1].copy()
    r0 = pkg.submit(ctx, kerns[0], p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                    max_iter=2000, precision=prec)
    r1 = pkg.submit(ctx, kerns[0], p.factors, bad_k, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                    max_iter=2000, precision=prec)
    r2 = pkg.submit(ctx, kerns[0], p.factors, unsorted_k, unsorted_o, unsorted_v, p.r, p.lam,
                    p.rho, tol, max_iter=2000, precision=prec, sorted_obs=True)
    r3 = pkg.submit(ctx, kerns[0], p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                    max_iter=2000, precision=prec)
    with pytest.raises(pkg.CphifiError) as e:
        r1.wait()
    assert e.value.status == pkg.E_INVALID_ARG and "out of range" in str(e.value)
    with pytest.raises(pkg.CphifiError) as e:
        r2.wait()
    assert e.value.status == pkg.E_INVALID_ARG and "not sorted" in str(e.value)
    for rq in (r0, r3):
        W, st = rq.wait()
        np.testing.assert_array_equal(W, alone[0][0])


def test_kernel_in_use_cannot_be_destroyed(pkg):
    ctx = pkg.Context(0)
    p, prec, tol = _problems()[1]
    dK, UK = np.linalg.eigh(p.K)
    k = ctx.kernel_create(p.n, UK, dK)
    rq = pkg.submit(ctx, k, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, tol,
                    max_iter=2000, precision=prec)
    with pytest.raises(pkg.CphifiError) as e:
        k.close()
    assert e.value.status == pkg.E_INVALID_ARG
    W, st = rq.wait()
    assert st["status"] == pkg.OK
    k.close()  # the request has completed: now it may go
    ctx.close()
