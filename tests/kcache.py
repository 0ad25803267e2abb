"""Host eigendecompositions of the kernel matrices the GPU tests hand to the
library (numpy.linalg.eigh; Eq. eigK is the caller's one-time setup), kept
for the life of the test process so that the n = 8000 kernel is decomposed
once however many tests use it."""
import hashlib

import numpy as np

_CACHE = {}


def eigh_cached(K):
    key = (K.shape, hashlib.sha1(np.ascontiguousarray(K[::97, ::89]).tobytes()).hexdigest())
    if key not in _CACHE:
        if len(_CACHE) >= 3:
            _CACHE.pop(next(iter(_CACHE)))
        _CACHE[key] = np.linalg.eigh(K)
    return _CACHE[key]
