"""Autotuner host logic: the coordinate search and the JSON cache (no GPU)."""
import json

from paper_2305_14306_gb300 import tuning


class FakeCtx:
    def __init__(self):
        self.t = {"spec_points": list(tuning.BASE_SPEC), "chunk_min": 64, "nblocks": 152, "small_points": 0}
        self.sets = 0

    def get_tuning(self):
        return dict(self.t, spec_points=list(self.t["spec_points"]))

    def set_tuning(self, spec_points=None, chunk_min=None, nblocks=None, small_points=None):
        self.sets += 1
        if spec_points is not None:
            self.t["spec_points"] = list(spec_points)
        if chunk_min is not None:
            self.t["chunk_min"] = int(chunk_min)
        if small_points is not None:
            self.t["small_points"] = int(small_points)


BEST_SPEC = [0, 8192, 131072]


def cost_of(ctx):
    # a made-up landscape with its minimum at one listed threshold choice and chunk 256
    sp = ctx.t["spec_points"]
    return sum(abs(a - b) for a, b in zip(sp, BEST_SPEC)) / 1e4 + abs(ctx.t["chunk_min"] - 256) / 100 + 1.0


def test_search_finds_the_minimum_and_caches(tmp_path):
    path = str(tmp_path / "c.json")
    ctx = FakeCtx()
    t, rep = tuning.autotune(ctx, None, "S64-N8388608-L2", "GB300", cache=path, timer=lambda: cost_of(ctx))
    assert t == {"spec_points": BEST_SPEC, "chunk_min": 256, "small_points": 0}
    assert ctx.t["spec_points"] == t["spec_points"] and ctx.t["chunk_min"] == 256
    assert rep["tuned_ms"] <= rep["default_ms"] and not rep["cached"]
    data = json.load(open(path))
    assert data["GB300|S64-N8388608-L2"]["tuning"] == t
    # a second process reads the cache and does not time anything
    ctx2 = FakeCtx()
    t2, rep2 = tuning.autotune(ctx2, None, "S64-N8388608-L2", "GB300", cache=path,
                               timer=lambda: (_ for _ in ()).throw(AssertionError("timed")))
    assert t2 == t and rep2["cached"] and ctx2.t["chunk_min"] == 256
    # another GPU name is another entry
    ctx3 = FakeCtx()
    tuning.autotune(ctx3, None, "S64-N8388608-L2", "other", cache=path, timer=lambda: cost_of(ctx3))
    assert set(json.load(open(path))) == {"GB300|S64-N8388608-L2", "other|S64-N8388608-L2"}


def test_default_kept_when_nothing_is_faster():
    ctx = FakeCtx()
    t, rep = tuning.autotune(ctx, None, "k", "g", cache=None, timer=lambda: 1.0)
    assert t == {"spec_points": list(tuning.BASE_SPEC), "chunk_min": 64, "small_points": 0}
    assert rep["tried"] == (1 + (len(tuning.SPEC_CHOICES) - 1) + (len(tuning.CHUNK_MINS) - 1)
                            + (len(tuning.SMALL_POINTS) - 1))


def test_signature_and_corrupt_cache(tmp_path):
    assert tuning.signature([20000] * 64, 2) == "S64-N1048576-L2"
    assert tuning.signature([1 << 20], 4) == "S1-N1048576-L4"
    assert tuning.signature([5, 5, 5], 1) == "S4-N16-L1"
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tuning.load_cache(str(bad)) == {}
    assert tuning.spec_for(0.0) == [0, 0, 0]
    assert tuning.spec_for(1e9)[2] == 1 << 31
    assert list(tuning.BASE_SPEC) in [list(c) for c in tuning.SPEC_CHOICES]
    for c in tuning.SPEC_CHOICES:
        assert c[0] <= c[1] <= c[2]
