"""Element-wise comparison used by the GPU parity tests.

For a computed n x r array `a` and the oracle's `b`, every element must satisfy

    |a_ij - b_ij| <= tol * (|b_ij| + max_k |b_ik|)

i.e. a relative bound per element, loosened only by the size of its own row
(one row per kernel index).  A row of the oracle that is exactly zero (a
kernel index with no observations) must come back exactly zero.  Unlike a
norm-wise check, a large error confined to a short row (an index with one or
two observations) cannot hide under the norm of the long rows.
"""
import json
import os

import numpy as np

# With CPHIFI_PARITY_LOG set, every check appends {what, tol, worst err/bound}
# to that file (one JSON object per line): the margins behind the tolerances.
_LOG = os.environ.get("CPHIFI_PARITY_LOG")


def check_rows(a, b, tol, what=""):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if b.ndim == 1:
        a, b = a[:, None], b[:, None]
    assert np.all(np.isfinite(a)), f"{what}: non-finite values"
    rowmax = np.max(np.abs(b), axis=1, keepdims=True) if b.shape[1] else np.zeros((b.shape[0], 1))
    bound = tol * (np.abs(b) + rowmax)
    err = np.abs(a - b)
    bad = err > bound
    if bad.any():
        i, j = np.argwhere(bad)[0]
        ratio = float(np.max(np.where(bound > 0, err / np.where(bound > 0, bound, 1), np.inf)))
        raise AssertionError(f"{what}: {int(bad.sum())} elements out of bound (tol {tol}); "
                             f"first at ({i}, {j}): got {a[i, j]!r}, want {b[i, j]!r}, "
                             f"row max {rowmax[i, 0]!r}; worst err/bound {ratio:.3g}")
    worst = float(np.max(err / np.maximum(np.abs(b) + rowmax, 1e-300))) if b.size else 0.0
    if _LOG:
        with open(_LOG, "a") as fh:
            fh.write(json.dumps({"what": what, "tol": tol, "worst_rel": worst,
                                 "margin": (tol / worst) if worst > 0 else None}) + "\n")
    return worst
