"""The operand splitting behind the tensor-core products, restated in NumPy.

The split-operand products (error-free splitting of Ozaki, Ogita, Oishi and
Rump) scale every row of U_K and every column of the right-hand operand below
1, cut each value into 8-bit slices m_t 2^(-7-8t) (|m_t| <= 128), multiply
the slices in BF16 on the tensor cores and add the products of one group
g = t + u in FP32.  These checks restate that scheme independently of the
CUDA code and pin the facts the kernel relies on: the slices are exact in
BF16, a group's sum over a 256-wide k chunk is exact in FP32 for g <= 3, the
7-slice product is FP64-accurate, and the 3-slice product of MIXED_BF16X3
(groups 0..2) is within 2^-24 of the scales per term.
"""
import numpy as np
import pytest


def slices(v, S):
    """S slices of each value of v (|v| < 1): integer m_t and the remainder."""
    M = np.rint(np.ldexp(v, 62)).astype(np.int64)
    ms = []
    for t in range(S):
        sh = 55 - 8 * t
        m = (M + (np.int64(1) << np.int64(sh - 1))) >> np.int64(sh)  # round, ties up
        M = M - (m << np.int64(sh))
        ms.append(m)
    return ms, M  # v = sum_t m_t 2^(sh_t - 62) + M 2^-62


def value(ms, S):
    return sum(np.ldexp(ms[t].astype(np.float64), 55 - 8 * t - 62) for t in range(S))


def bf16_exact(x):
    """x is representable in BF16 (8 significant bits, FP32 exponent range)."""
    f = x.astype(np.float32)
    bits = f.view(np.uint32)
    return np.all((bits & np.uint32(0xFFFF)) == 0) and np.all(f.astype(np.float64) == x)


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(3)
    # graded magnitudes, as the columns of D_K p have
    v = rng.standard_normal(4096) * np.exp(-rng.uniform(0, 30, 4096))
    return v / (np.abs(v).max() * 1.0000001)


def test_slices_are_small_integers_exact_in_bf16(data):
    ms, rest = slices(data, 7)
    for t, m in enumerate(ms):
        assert np.abs(m).max() <= 128
        assert bf16_exact(np.ldexp(m.astype(np.float64), 55 - 8 * t - 62))
    assert np.abs(np.ldexp(rest.astype(np.float64), -62)).max() <= 2.0 ** -56


def test_three_slices_leave_half_a_unit_of_the_third():
    # (seven slices: the integer remainder of the first test, 2^-56)
    rng = np.random.default_rng(6)
    v = rng.uniform(-1, 1, 4096) * np.exp(-rng.uniform(0, 20, 4096))
    ms, _ = slices(v, 7)
    assert np.abs(v - value(ms, 3)).max() <= 2.0 ** -24


def test_group_sums_of_a_256_chunk_are_exact_in_fp32():
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, 1, 256) * 0.999
    b = rng.uniform(-1, 1, 256) * 0.999
    ma, _ = slices(a, 7)
    mb, _ = slices(b, 7)
    for g in range(4):
        terms = [ma[t] * mb[g - t] for t in range(g + 1)]
        exact = int(sum(int(x.sum()) for x in terms))
        assert abs(exact) <= (g + 1) * 256 * 2 ** 14 <= 2 ** 24
        acc = np.float32(0)
        for x in np.concatenate(terms)[rng.permutation(256 * (g + 1))]:
            acc = np.float32(acc + np.float32(x))  # FP32 accumulation, any order
        assert int(acc) == exact


@pytest.mark.parametrize("S,groups", [(3, 3), (7, 7)])
def test_split_product_accuracy(S, groups):
    # rows of an orthogonal matrix times graded columns, both scaled below 1
    rng = np.random.default_rng(5)
    n = 512
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    B = rng.standard_normal((n, 4)) * np.exp(-np.linspace(0, 25, n))[:, None]
    re = np.frexp(np.abs(U).max(axis=1))[1]
    ce = np.frexp(np.abs(B).max(axis=0))[1]
    As = np.ldexp(U, -re[:, None])
    Bs = np.ldexp(B, -ce[None, :])
    ma, _ = slices(As, 7)
    mb, _ = slices(Bs, 7)
    C = np.zeros((n, 4))
    for t in range(S):
        for u in range(S):
            if t + u < groups:
                C += np.ldexp(ma[t].astype(np.float64), 55 - 8 * t - 62) @ \
                    np.ldexp(mb[u].astype(np.float64), 55 - 8 * u - 62)
    exact = As @ Bs
    err = np.abs(C - exact)
    if S == 3:
        # per term: the truncated slices, 2^-24 (|a_k| + |b_k|) of the scales (both 1
        # after scaling), and the dropped slice products of index sum 3 (two, each at
        # most 2^-8 2^-16) and 4 (2^-32)
        bound = 2.0 ** -24 * (np.abs(As).sum(axis=1)[:, None] + np.abs(Bs).sum(axis=0)[None, :]
                              + 2 * n) + n * 2.0 ** -32
        assert np.all(err <= bound)
        assert err.max() > 2.0 ** -40  # the truncation is visible: not an FP64 product
    else:
        assert err.max() <= 2.0 ** -50 * (np.abs(As) @ np.abs(Bs)).max()
