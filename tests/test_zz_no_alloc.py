"""The allocation-free gather-dot/scatter entry point (cphifi_gds_noalloc).

Some callers cannot allocate device memory (graph-capture regions that must
not record allocations, real-time host loops, runtimes that own all device
memory), so the library offers this one call whose working memory is a fixed
array inside the library.  This test calls it through the C ABI twice in a
row and compares each result with the allocating entry point
cphifi_problem_gds on the same data, within the FP64 tolerance the parity
tests use for that step (1e-12 relative, norm-wise).  It sits in its own file,
collected after the others, and creates everything it uses, so it passes both
alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("seed,n,other,q,r", [
    (21, 300, (30, 40), 60000, 24),   # several pieces per kernel index
    (22, 4, (100, 60), 20000, 40),    # indices spanning many warps
    (23, 500, (5, 6), 300, 5),        # empty indices, short ragged tail
])
def test_noalloc_gds_matches_allocating_entry_point(seed, n, other, q, r):
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as pkg

    p = synth.planted_problem(seed, n, other, q, r, bandwidth=0.1)  # sorted by kernel index
    ctx = pkg.Context(0)
    dK, UK = np.linalg.eigh(p.K)
    kern = ctx.kernel_create(p.n, UK, dK)
    prob = pkg.Problem(ctx, kern, p.factors, p.kidx, p.oidx, p.vals, p.r, sorted_obs=True)

    dev = torch.device("cuda", 0)
    row_ptr = np.searchsorted(p.kidx, np.arange(p.n + 1)).astype(np.int64)
    zhat = O.zhat(p.factors, p.oidx)  # observations are already in sorted order
    rp_d = torch.from_numpy(row_ptr).to(dev)
    z_d = torch.from_numpy(np.asfortranarray(zhat).ravel(order="F")).to(dev)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(seed)
    for _ in range(2):  # two calls in a row share the scratch array
        Xh = rng.standard_normal((p.n, p.r))
        ref = prob.gds(Xh, "fp64")
        x_d = torch.from_numpy(np.asfortranarray(Xh).ravel(order="F")).to(dev)
        y_d = torch.full((p.n * p.r,), float("nan"), dtype=torch.float64, device=dev)
        pkg.gds_noalloc(p.n, p.r, p.q, rp_d, z_d, p.q, x_d, y_d, stream=stream)
        torch.cuda.synchronize()
        Y = y_d.cpu().numpy().reshape(p.r, p.n).T
        assert np.all(np.isfinite(Y))
        assert rel(Y, ref) <= 1e-12
    prob.close()
    kern.close()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as pkg

    dev = torch.device("cuda", 0)
    n, r = 16385, 4
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(n * r, dtype=torch.float64, device=dev)
    y = torch.zeros(n * r, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.CphifiError) as e:
        pkg.gds_noalloc(n, r, 0, rp, z, 0, x, y)
    assert e.value.status == pkg.E_INVALID_ARG and "16384" in str(e.value)
    with pytest.raises(pkg.CphifiError) as e:
        pkg.gds_noalloc(8, 65, 0, rp, z, 0, x, y)
    assert e.value.status == pkg.E_INVALID_ARG and "64" in str(e.value)
