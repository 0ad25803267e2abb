"""Launch shapes per size bucket (cphifi_ctx_set_tuning) and the autotuner.

Shapes change only how the work is cut (gather-dot/scatter warps, product
k-splits), so a solve with any accepted shapes must still meet the oracle's
gates (FP64 true residual <= tol, fitted values within 10 tol), give the
same bits every time, and give the same bits submitted as one-shot.
"""
import json

import numpy as np
import pytest

import oracle as O
import synth
from kcache import eigh_cached

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as p
    return p


@pytest.mark.parametrize("shapes", [{"gds_warps_per_sm": 4, "split32": 3},
                                    {"gds_warps_per_sm": 32, "split32": 1, "split_wide": 2},
                                    {"split32": 64, "split_wide": 64}])
def test_tuned_shapes_keep_results_and_determinism(pkg, shapes):
    p = synth.workload("c1_fp64_n100_q6e3_r5", seed=3)
    ctx = pkg.Context(0)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    ctx.set_tuning(pkg.size_bucket(p.n, p.q, p.r), shapes)
    W1, s1 = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-8,
                       2000, precision="mixed_fp32", sorted_obs=True)
    W2, s2 = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-8,
                       2000, precision="mixed_fp32", sorted_obs=True)
    np.testing.assert_array_equal(W1, W2)
    W3, s3 = pkg.submit(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-8,
                        2000, precision="mixed_fp32", sorted_obs=True).wait()
    np.testing.assert_array_equal(W1, W3)
    res = O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W1)
    assert s1["status"] == 0 and res <= 1e-8, (res, s1)
    Wd = O.solve_direct(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho)
    Zh = O.zhat(p.factors, p.oidx)
    fw = O.fitted_values(p.K, Wd, p.kidx, Zh)
    assert np.linalg.norm(O.fitted_values(p.K, W1, p.kidx, Zh) - fw) <= 1e-7 * np.linalg.norm(fw)
    kern.close()
    ctx.close()


def test_bad_tuning_rejected(pkg):
    ctx = pkg.Context(0)
    with pytest.raises(pkg.CphifiError):
        ctx.set_tuning((6, 12, 5), {"split32": 65})
    with pytest.raises(pkg.CphifiError):
        ctx.set_tuning((6, 12, 0), {"split32": 2})
    ctx.set_tuning((6, 12, 5), {"split32": 2})
    ctx.set_tuning((6, 12, 5), None)
    ctx.close()


def test_autotuner_picks_shapes_and_caches_them(pkg, tmp_path):
    from paper_2603_25691_gb300 import autotune
    p = synth.planted_problem(31, 300, (30, 40), 40000, 16, bandwidth=0.1)
    ctx = pkg.Context(0)
    dK, UK = eigh_cached(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    inst = dict(factors=p.factors, kidx=p.kidx, oidx=p.oidx, vals=p.vals, r=p.r, lam=p.lam,
                rho=p.rho, sorted=True)
    path = str(tmp_path / "tuning.json")
    cache = autotune.Cache(path)
    assert cache.tune_instances(ctx, [(kern, inst)], "mixed_fp32", iters=4, reps=1) == 1
    with open(path) as fh:
        saved = json.load(fh)
    (key, shapes), = saved.items()
    assert key == "mixed_fp32 %d %d %d" % pkg.size_bucket(p.n, p.q, p.r)
    assert shapes["gds_warps_per_sm"] in autotune.GDS_WARPS_PER_SM
    assert shapes["split32"] in autotune.SPLITS
    assert autotune.Cache(path).apply(ctx, "mixed_fp32") == 1
    W, st = pkg.solve(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, p.lam, p.rho, 1e-8,
                      2000, precision="mixed_fp32", sorted_obs=True)
    assert st["status"] == 0
    assert O.relative_residual(p.K, p.factors, p.kidx, p.oidx, p.vals, p.lam, p.rho, W) <= 1e-8
    kern.close()
    ctx.close()
