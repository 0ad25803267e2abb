"""Host logic of the launch-shape autotuner (no GPU): buckets, the JSON cache,
and what apply() hands to the context.  The timing itself (tune) is replaced
by a stand-in; its GPU side is covered by tests/test_gpu_tuning.py."""
import json

import paper_2603_25691_gb300 as pkg
from paper_2603_25691_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.tuning = {}

    def set_tuning(self, bucket, shapes):
        self.tuning[tuple(bucket)] = shapes


class FakeKernel:
    def __init__(self, n):
        self.n = n


def _inst(q, r):
    return dict(kidx=[0] * q, r=r)


def test_size_bucket():
    assert pkg.size_bucket(1000, 5000, 16) == (9, 12, 16)
    assert pkg.size_bucket(1024, 4096, 16) == (10, 12, 16)
    assert pkg.size_bucket(50, 0, 4) == (5, 0, 4)


def test_cache_tunes_each_bucket_once_and_applies_only_launch_shapes(tmp_path, monkeypatch):
    calls = []

    def fake_tune(ctx, kernel, inst, precision, **kw):
        calls.append((kernel.n, len(inst["kidx"]), inst["r"], precision))
        if kernel.n == 99:
            raise pkg.CphifiError(pkg.E_UNSUPPORTED, "not tunable")
        return {"gds_warps_per_sm": 8, "split32": 4, "gds_ms": {"8": 0.1},
                "product_ms": {"4": 0.2}, "n": kernel.n, "q": len(inst["kidx"])}

    monkeypatch.setattr(autotune, "tune", fake_tune)
    path = tmp_path / "shapes.json"
    cache = autotune.Cache(str(path))
    insts = [(FakeKernel(1000), _inst(5000, 16)),   # bucket (9, 12, 16)
             (FakeKernel(1020), _inst(6000, 16)),   # same bucket: not tuned again
             (FakeKernel(1000), _inst(5000, 32)),   # another rank: another bucket
             (FakeKernel(99), _inst(10, 4))]        # the tuner fails: skipped, not cached
    assert cache.tune_instances(FakeCtx(), insts, "mixed_fp32") == 2
    assert [c[0] for c in calls] == [1000, 1000, 99]
    assert sorted(cache.entries) == ["mixed_fp32 9 12 16", "mixed_fp32 9 12 32"]
    # the file holds the same entries; a second pass over the instances tunes nothing
    assert json.loads(path.read_text()) == cache.entries
    again = autotune.Cache(str(path))
    assert again.tune_instances(FakeCtx(), insts[:3], "mixed_fp32") == 0
    # apply: the integer launch shapes of the requested precision only
    ctx = FakeCtx()
    assert again.apply(ctx, "mixed_fp32") == 2
    assert ctx.tuning == {(9, 12, 16): {"gds_warps_per_sm": 8, "split32": 4},
                          (9, 12, 32): {"gds_warps_per_sm": 8, "split32": 4}}
    assert again.apply(FakeCtx(), "mixed_bf16x3") == 0


def test_every_precision_has_a_product_split_field():
    # the field tune() varies for the products is one the context accepts
    assert set(autotune.PRODUCT_SPLIT_FIELD) == set(pkg.PRECISIONS)
    assert set(autotune.PRODUCT_SPLIT_FIELD.values()) <= {f for f, _ in pkg.Tuning._fields_}
