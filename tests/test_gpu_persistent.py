"""Many mixed-FP32 solves in one persistent launch (cphifi_solve_batch),
against the FP64 oracle.

Every solve of the launch is gated by the oracle's FP64 true residual
(relative residual <= tol, the solve's own stopping rule), each result must
be bitwise the same alone and in the mix (the launch's tiles add their
partial sums in a fixed order whatever block runs them), and bad inputs or a
too small max_iter fail only their own item.
"""
import numpy as np
import pytest

import oracle as O
import synth
from kcache import eigh_cached

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as p
    return p


# (seed, n, other sizes, q, r, kernel, shuffled): ranks 1..64, several tiles
# and ragged tails in every phase, an index range with empty kernel rows, one
# instance with fewer observations than unknowns.
MIX = [
    (51, 100, (20, 30), 6000, 5, "gaussian", True),
    (52, 300, (30, 40), 40000, 16, "matern32", False),
    (53, 64, (5, 6, 7), 9000, 16, "gaussian", True),
    (54, 120, (25, 25), 20000, 40, "gaussian", False),
    (55, 50, (12, 14), 4000, 64, "matern32", True),
    (56, 457, (60, 70), 60000, 32, "gaussian", False),
    (57, 30, (10,), 200, 1, "gaussian", True),
    (58, 700, (3, 4), 500, 7, "matern32", False),
    (59, 1223, (40, 50), 30000, 8, "gaussian", False),
]
TOL = 1e-6
LAM, RHO = 1e-4, 1e-6


def _problems():
    out = []
    for seed, n, other, q, r, kern, shuf in MIX:
        out.append(synth.planted_problem(seed, n, other, q, r, kernel=kern, bandwidth=0.1,
                                         lam=LAM, rho=RHO, shuffle=shuf))
    return out


@pytest.fixture(scope="module")
def env(pkg):
    ctx = pkg.Context(0)
    probs = _problems()
    kerns = []
    for p in probs:
        dK, UK = eigh_cached(p.K)
        kerns.append(ctx.kernel_create(p.n, UK, dK))
    yield ctx, probs, kerns
    for k in kerns:
        k.close()
    ctx.close()


def _items(probs, kerns):
    return [dict(kernel=k, factors=p.factors, kidx=p.kidx, oidx=p.oidx, vals=p.vals, r=p.r)
            for p, k in zip(probs, kerns)]


def test_every_solve_meets_tol_against_the_oracle(pkg, env):
    ctx, probs, kerns = env
    Ws, stats, info = pkg.solve_batch(ctx, _items(probs, kerns), LAM, RHO, TOL, max_iter=4000)
    assert info["blocks"] >= 1 and info["timed_out"] == 0
    assert info["tiles"] > 0 and info["kernel_ms"] > 0
    for W, st, p in zip(Ws, stats, probs):
        assert st["status"] == pkg.OK, st
        assert st["kernel_launches"] == 1
        assert st["true_residuals"] >= 1 and st["rel_residual"] <= TOL
        res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
        assert res <= TOL, (p.n, p.r, res)


def test_results_are_the_same_alone_and_in_the_mix(pkg, env):
    ctx, probs, kerns = env
    items = _items(probs, kerns)
    Wmix, smix, _ = pkg.solve_batch(ctx, items, LAM, RHO, TOL, max_iter=4000)
    # another order and a subset: the same bits per problem
    perm = [4, 0, 8, 2]
    Wsub, ssub, _ = pkg.solve_batch(ctx, [items[k] for k in perm], LAM, RHO, TOL, max_iter=4000)
    for j, k in enumerate(perm):
        np.testing.assert_array_equal(Wsub[j], Wmix[k])
        assert ssub[j]["iterations"] == smix[k]["iterations"]
    for k in (1, 6):
        Walone, salone, _ = pkg.solve_batch(ctx, [items[k]], LAM, RHO, TOL, max_iter=4000)
        np.testing.assert_array_equal(Walone[0], Wmix[k])
        assert salone[0]["true_residuals"] == smix[k]["true_residuals"]


def test_uneven_batch_sample(pkg):
    # instances drawn as in the 256-solve uneven batch (n log-uniform on
    # [50, 2000], q log-uniform, r in {4, 8, 16, 32}, Gaussian or Matern),
    # limited to sizes the oracle checks in seconds
    specs = [s for s in synth.batch_specs(7, 64) if s["n"] <= 600 and s["q"] <= 60000][:12]
    assert len(specs) >= 8
    ctx = pkg.Context(0)
    try:
        probs = [synth.batch_problem(s, LAM, RHO) for s in specs]
        kerns = []
        for p in probs:
            dK, UK = eigh_cached(p.K)
            kerns.append(ctx.kernel_create(p.n, UK, dK))
        Ws, stats, info = pkg.solve_batch(ctx, _items(probs, kerns), LAM, RHO, TOL,
                                          max_iter=6000)
        for W, st, p in zip(Ws, stats, probs):
            assert st["status"] == pkg.OK, st
            res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W)
            assert res <= TOL, (p.n, p.r, res)
        for k in kerns:
            k.close()
    finally:
        ctx.close()


def test_device_inputs_and_outputs(pkg, env):
    import torch
    ctx, probs, kerns = env
    dev = torch.device("cuda", 0)
    items_h = _items(probs[:4], kerns[:4])
    Wh, _, _ = pkg.solve_batch(ctx, items_h, LAM, RHO, TOL, max_iter=4000)
    items_d = []
    for p, k in zip(probs[:4], kerns[:4]):
        f = [torch.from_numpy(np.asfortranarray(F).ravel(order="F")).to(dev) for F in p.factors]
        items_d.append(dict(kernel=k, factors=f,
                            kidx=torch.from_numpy(p.kidx.astype(np.int32)).to(dev),
                            oidx=torch.from_numpy(np.ascontiguousarray(p.oidx, dtype=np.int32)).to(dev),
                            vals=torch.from_numpy(p.vals).to(dev), r=p.r))
    Wd, sd, _ = pkg.solve_batch(ctx, items_d, LAM, RHO, TOL, max_iter=4000)
    for W, Wref, p in zip(Wd, Wh, probs[:4]):
        np.testing.assert_array_equal(W.cpu().numpy().reshape(p.r, p.n).T, Wref)


def test_bad_inputs_and_max_iter_fail_their_item_only(pkg, env):
    ctx, probs, kerns = env
    items = _items(probs[:3], kerns[:3])
    Wref, _, _ = pkg.solve_batch(ctx, items, LAM, RHO, TOL, max_iter=4000)
    p = probs[1]
    bad = dict(items[1])
    bad_k = p.kidx.copy()
    bad_k[len(bad_k) // 2] = p.n + 3
    bad["kidx"] = bad_k
    Ws, stats, info = pkg.solve_batch(ctx, [items[0], bad, items[2]], LAM, RHO, TOL,
                                      max_iter=4000)
    assert stats[1]["status"] == pkg.E_INVALID_ARG
    for k in (0, 2):
        assert stats[k]["status"] == pkg.OK
        np.testing.assert_array_equal(Ws[k], Wref[k])
    # max_iter reached: not converged, never more iterations than allowed
    Ws, stats, _ = pkg.solve_batch(ctx, items, LAM, RHO, 1e-14, max_iter=3)
    for st in stats:
        assert st["status"] == pkg.E_NOT_CONVERGED and st["iterations"] <= 3


def test_unsupported_and_bad_arguments(pkg, env):
    ctx, probs, kerns = env
    items = _items(probs[:2], kerns[:2])
    with pytest.raises(pkg.CphifiError) as e:
        pkg.solve_batch(ctx, items, LAM, RHO, TOL, precision="fp64")
    assert e.value.status == pkg.E_UNSUPPORTED
    with pytest.raises(pkg.CphifiError) as e:
        pkg.solve_batch(ctx, items, LAM, -1.0, TOL)
    assert e.value.status == pkg.E_INVALID_ARG
    Ws, stats, info = pkg.solve_batch(ctx, [], LAM, RHO, TOL)
    assert Ws == [] and stats == []


def test_bounded_wait_expires_for_a_held_item(pkg, env):
    # A held item is created but never started, so the launch can end only by
    # its bounded idle wait: the held item reports a timeout, the others their
    # own results, bit for bit, and the context stays usable.
    ctx, probs, kerns = env
    items = _items(probs[:2], kerns[:2])
    Wref, _, _ = pkg.solve_batch(ctx, items, LAM, RHO, TOL, max_iter=4000)
    for bad in (0, 600001, -5):
        with pytest.raises(pkg.CphifiError) as e:
            ctx.set_batch_wait(bad)
        assert e.value.status == pkg.E_INVALID_ARG
    ctx.set_batch_wait(100)
    try:
        held = dict(items[1], hold=True)
        Ws, stats, info = pkg.solve_batch(ctx, [items[0], held], LAM, RHO, TOL, max_iter=4000)
        assert info["timed_out"] == 1
        assert stats[0]["status"] == pkg.OK
        np.testing.assert_array_equal(Ws[0], Wref[0])
        assert stats[1]["status"] == pkg.E_TIMEOUT and stats[1]["iterations"] == 0
        # the launch waited about the bound, not the 4 s default
        assert 100.0 <= info["kernel_ms"] < 2000.0, info
    finally:
        ctx.set_batch_wait(4000)
    Ws, stats, info = pkg.solve_batch(ctx, items, LAM, RHO, TOL, max_iter=4000)
    assert info["timed_out"] == 0
    for k in (0, 1):
        assert stats[k]["status"] == pkg.OK
        np.testing.assert_array_equal(Ws[k], Wref[k])
