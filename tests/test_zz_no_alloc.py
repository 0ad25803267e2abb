"""The allocation-free gather-dot/scatter entry point (cphifi_gds_noalloc).

Some callers cannot allocate device memory (a real-time host loop that may
not take the allocator's locks or wait for its implicit synchronisation, a
runtime that owns all device memory), so the library offers this one call
whose working memory is a fixed array inside the library.  This test calls it
through the C ABI twice in a row on the same data and checks each result
against the FP64 oracle (Eqs. vl and yhat1: scatter_rows of gather_dot) and
against the allocating entry point cphifi_problem_gds, element by element
within the FP64 bound of the other parity tests.  It also checks that a call
leaves the device's free memory unchanged, and that a row pointer that is not
a CSR of q entries is caught on the device (Y1 comes back as NaN, nothing
else is written).  It sits in its own file, collected after the others, and
creates everything it uses, so it passes both alone in a fresh process and
after the rest of the suite.
"""
import numpy as np
import pytest

import oracle as O
import synth
from elementwise import check_rows

pytestmark = pytest.mark.gpu


def _pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2603_25691_gb300 as pkg
    return pkg


@pytest.mark.parametrize("seed,n,other,q,r", [
    (21, 300, (30, 40), 60000, 24),   # several pieces per kernel index
    (22, 4, (100, 60), 20000, 40),    # indices spanning many warps
    (23, 500, (5, 6), 300, 5),        # empty indices, short ragged tail
    (24, 200, (20, 25), 7000, 13),    # 9 <= r <= 16
])
def test_noalloc_gds_matches_oracle_and_allocating_entry_point(seed, n, other, q, r):
    import torch

    pkg = _pkg()
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
    for call in range(2):  # two calls in a row share the scratch array
        Xh = rng.standard_normal((p.n, p.r))
        ref = O.scatter_rows(p.n, p.kidx, O.gather_dot(Xh, p.kidx, zhat), zhat)
        x_d = torch.from_numpy(np.asfortranarray(Xh).ravel(order="F")).to(dev)
        y_d = torch.full((p.n * p.r,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        pkg.gds_noalloc(p.n, p.r, p.q, rp_d, z_d, p.q, x_d, y_d, stream=stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(0)[0]
        if call == 1:  # (the first call may load the library's kernels)
            assert free1 == free0, (free0, free1)
        Y = y_d.cpu().numpy().reshape(p.r, p.n).T
        check_rows(Y, ref, 1e-12, "noalloc vs oracle")
        check_rows(Y, prob.gds(Xh, "fp64"), 1e-12, "noalloc vs cphifi_problem_gds")
    prob.close()
    kern.close()
    ctx.close()


def test_noalloc_bad_row_pointer_gives_nan():
    import torch

    pkg = _pkg()
    dev = torch.device("cuda", 0)
    n, r, q = 6, 3, 10
    z = torch.ones(q * r, dtype=torch.float64, device=dev)
    x = torch.ones(n * r, dtype=torch.float64, device=dev)
    good = torch.tensor([0, 2, 2, 5, 7, 9, 10], dtype=torch.int64, device=dev)
    y = torch.zeros(n * r, dtype=torch.float64, device=dev)
    pkg.gds_noalloc(n, r, q, good, z, q, x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    for bad in ([1, 2, 2, 5, 7, 9, 10],         # row_ptr[0] != 0
                [0, 2, 2, 5, 7, 9, 9],          # row_ptr[n] != q
                [0, 5, 2, 5, 7, 9, 10]):        # decreasing
        y = torch.zeros(n * r, dtype=torch.float64, device=dev)
        pkg.gds_noalloc(n, r, q, torch.tensor(bad, dtype=torch.int64, device=dev), z, q, x, y)
        torch.cuda.synchronize()
        assert torch.isnan(y).all(), bad
    # a good call after the bad ones: the error word is cleared again
    y = torch.zeros(n * r, dtype=torch.float64, device=dev)
    pkg.gds_noalloc(n, r, q, good, z, q, x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    pkg = _pkg()
    dev = torch.device("cuda", 0)
    n, r = 16385, 4
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(n * r, dtype=torch.float64, device=dev)
    y = torch.zeros(n * r, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.CphifiError) as e:
        pkg.gds_noalloc(n, r, 0, rp, z, 0, x, y)
    assert e.value.status == pkg.E_INVALID_ARG and "16384" in str(e.value)
    rp9 = torch.zeros(9, dtype=torch.int64, device=dev)
    with pytest.raises(pkg.CphifiError) as e:
        pkg.gds_noalloc(8, 65, 0, rp9, z, 0, torch.zeros(8 * 65, dtype=torch.float64, device=dev),
                        torch.zeros(8 * 65, dtype=torch.float64, device=dev))
    assert e.value.status == pkg.E_INVALID_ARG and "64" in str(e.value)
    with pytest.raises(ValueError):  # int32 row pointer: refused before the call
        pkg.gds_noalloc(8, 2, 0, rp9.to(torch.int32), z, 0, x, y)
