"""Autotuner of the solver's launch shapes per problem-size bucket.

The launch shapes that depend on the problem's size -- how many warps the
gather-dot/scatter (Eqs. vl, yhat1) spreads its observation ranges over, and
how many pieces the k range of each n x n product (§4.4.1) is split into --
come from heuristics in the library.  For a bucket (floor(log2 n),
floor(log2 q), r) this module times candidate shapes on a representative
problem of the bucket and keeps the fastest:

* gather-dot/scatter warps per SM in GDS_WARPS_PER_SM, timed by the
  library's own CUDA events around each gather-dot/scatter launch (solve
  statistics with profile = 1);
* then, with that choice, the splits of the products the precision uses
  (FP32 SIMT, tensor-core, FP64-accurate), timed the same way around each
  product launch.

Each candidate is a fresh problem created with the candidate's shapes set on
the context (cphifi_ctx_set_tuning) and a fixed number of PCG iterations.
Results are cached as JSON ({"mixed_fp32 11 20 40": {"gds_warps_per_sm": 8,
...}}) and loaded into a context with apply().  Tuning changes only launch
shapes: results stay deterministic for a given context and problem.
"""
from __future__ import annotations

import json
import os

from . import CphifiError, Problem, size_bucket

GDS_WARPS_PER_SM = (4, 8, 16, 24, 32)
SPLITS = (1, 2, 4, 8, 12, 16, 24, 32)
# the tuning field of the products each operator arithmetic runs
PRODUCT_SPLIT_FIELD = {"mixed_fp32": "split32", "mixed_tf32": "split_tc", "mixed_bf16": "split_tc",
                       "mixed_tf32x3": "split_tc", "mixed_bf16x3": "split_wide",
                       "fp64_emulated": "split_wide", "fp64": "split64"}


def _key(precision: str, bucket) -> str:
    return f"{precision} {bucket[0]} {bucket[1]} {bucket[2]}"


def _time(ctx, kernel, inst, precision, shapes, iters, reps):
    """Per-launch milliseconds (gather-dot/scatter, products) of a solve of
    `iters` iterations with the given shapes, the best of `reps` runs."""
    bucket = size_bucket(kernel.n, len(inst["kidx"]), inst["r"])
    ctx.set_tuning(bucket, shapes)
    try:
        prob = Problem(ctx, kernel, inst["factors"], inst["kidx"], inst["oidx"], inst["vals"],
                       inst["r"], sorted_obs=inst.get("sorted", False),
                       lowp=precision != "fp64")
        best_g, best_p = float("inf"), float("inf")
        for _ in range(reps + 1):  # the first run warms up
            _, st = prob.solve(inst["lam"], inst["rho"], 1e-30, iters, precision=precision,
                               profile=True, raise_on_error=False)
            if st["gds_launches"]:
                best_g = min(best_g, st["gds_ms"] / st["gds_launches"])
            if st["gemm_launches"]:
                best_p = min(best_p, st["gemm_ms"] / st["gemm_launches"])
        prob.close()
    finally:
        ctx.set_tuning(bucket, None)
    return best_g, best_p


def tune(ctx, kernel, inst, precision="mixed_fp32", iters=6, reps=2) -> dict:
    """Shapes for the bucket of one representative problem `inst` (a dict
    with factors, kidx, oidx, vals, r, lam, rho and optionally sorted)."""
    n, q = kernel.n, len(inst["kidx"])
    times = {}
    for w in GDS_WARPS_PER_SM:
        times[w] = _time(ctx, kernel, inst, precision, {"gds_warps_per_sm": w}, iters, reps)[0]
    wbest = min(times, key=times.get)
    f = PRODUCT_SPLIT_FIELD[precision]
    ptimes = {}
    for s_ in [s for s in SPLITS if s <= max(1, (n + 31) // 32)]:
        ptimes[s_] = _time(ctx, kernel, inst, precision, {"gds_warps_per_sm": wbest, f: s_},
                           iters, reps)[1]
    sbest = min(ptimes, key=ptimes.get)
    return {"gds_warps_per_sm": int(wbest), f: int(sbest),
            "gds_ms": {str(k): v for k, v in times.items()},
            "product_ms": {str(k): v for k, v in ptimes.items()}, "n": n, "q": q}


class Cache:
    """Tuned shapes per (precision, bucket), kept in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as fh:
                self.entries = json.load(fh)

    def save(self):
        if self.path:
            with open(self.path, "w") as fh:
                json.dump(self.entries, fh, indent=1, sort_keys=True)

    def tune_instances(self, ctx, instances, precision="mixed_fp32", **kw) -> int:
        """Tunes every bucket of `instances` (pairs (kernel, inst)) that the
        cache does not hold yet, on the bucket's first instance; returns how
        many buckets were tuned."""
        done = 0
        for kernel, inst in instances:
            key = _key(precision, size_bucket(kernel.n, len(inst["kidx"]), inst["r"]))
            if key in self.entries:
                continue
            try:
                self.entries[key] = tune(ctx, kernel, inst, precision, **kw)
            except CphifiError:
                continue
            done += 1
        self.save()
        return done

    def apply(self, ctx, precision="mixed_fp32") -> int:
        """Loads the cached shapes of `precision` into the context."""
        k = 0
        for key, shapes in self.entries.items():
            prec, a, b, c = key.split()
            if prec == precision:
                ctx.set_tuning((int(a), int(b), int(c)),
                               {f: v for f, v in shapes.items() if isinstance(v, int)
                                and f in ("gds_warps_per_sm", "split32", "split_tc",
                                          "split_wide", "split64")})
                k += 1
        return k
