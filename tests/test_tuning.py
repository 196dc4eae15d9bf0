"""Autotuner host logic: the coordinate search and the JSON cache (no GPU)."""
import json

from paper_2305_14306_gb300 import tuning


class FakeCtx:
    def __init__(self, refuse_clusters=False):
        self.t = {"spec_points": list(tuning.BASE_SPEC), "chunk_min": 64, "nblocks": 152, "small_points": 0,
                  "table_log2": 1, "pass_shape": 0}
        self.sets = 0
        self.refuse_clusters = refuse_clusters

    def get_tuning(self):
        return dict(self.t, spec_points=list(self.t["spec_points"]))

    def set_tuning(self, spec_points=None, chunk_min=None, nblocks=None, small_points=None, table_log2=None,
                   pass_shape=None):
        if small_points and self.refuse_clusters:
            raise RuntimeError("no cluster launch on this device")
        self.sets += 1
        if spec_points is not None:
            self.t["spec_points"] = list(spec_points)
        if chunk_min is not None:
            self.t["chunk_min"] = int(chunk_min)
        if small_points is not None:
            self.t["small_points"] = int(small_points)
        if table_log2 is not None:
            self.t["table_log2"] = int(table_log2)
        if pass_shape is not None:
            self.t["pass_shape"] = int(pass_shape)


BEST_SPEC = [0, 8192, 131072]


def cost_of(ctx):
    # a made-up landscape with its minimum at one listed threshold choice, chunk
    # 256, load factor 2^2 and pass shape 1
    sp = ctx.t["spec_points"]
    return (sum(abs(a - b) for a, b in zip(sp, BEST_SPEC)) / 1e4 + abs(ctx.t["chunk_min"] - 256) / 100
            + abs(ctx.t["table_log2"] - 2) * 0.3 + (0.0 if ctx.t["pass_shape"] == 1 else 0.2) + 1.0)


def test_search_finds_the_minimum_and_caches(tmp_path):
    path = str(tmp_path / "c.json")
    ctx = FakeCtx()
    t, rep = tuning.autotune(ctx, None, "S64-N8388608-L2", "GB300", cache=path, timer=lambda: cost_of(ctx))
    assert t == {"spec_points": BEST_SPEC, "chunk_min": 256, "small_points": 0, "table_log2": 2, "pass_shape": 1}
    assert ctx.t["spec_points"] == t["spec_points"] and ctx.t["chunk_min"] == 256
    assert ctx.t["table_log2"] == 2 and ctx.t["pass_shape"] == 1
    assert rep["tuned_ms"] <= rep["default_ms"] and not rep["cached"]
    data = json.load(open(path))
    assert data["GB300|S64-N8388608-L2"]["tuning"] == t
    # a second process reads the cache and does not time anything
    ctx2 = FakeCtx()
    t2, rep2 = tuning.autotune(ctx2, None, "S64-N8388608-L2", "GB300", cache=path,
                               timer=lambda: (_ for _ in ()).throw(AssertionError("timed")))
    assert t2 == t and rep2["cached"] and ctx2.t["chunk_min"] == 256 and ctx2.t["table_log2"] == 2
    # another GPU name is another entry
    ctx3 = FakeCtx()
    tuning.autotune(ctx3, None, "S64-N8388608-L2", "other", cache=path, timer=lambda: cost_of(ctx3))
    assert set(json.load(open(path))) == {"GB300|S64-N8388608-L2", "other|S64-N8388608-L2"}


def test_default_kept_when_nothing_is_faster():
    ctx = FakeCtx()
    t, rep = tuning.autotune(ctx, None, "k", "g", cache=None, timer=lambda: 1.0)
    assert t == {"spec_points": list(tuning.BASE_SPEC), "chunk_min": 64, "small_points": 0, "table_log2": 1,
                 "pass_shape": 0}
    assert rep["tried"] == 1 + sum(len(choices) - 1 for _, choices in tuning.STAGES)


def test_refused_settings_are_skipped_and_old_cache_entries_fill_defaults(tmp_path):
    ctx = FakeCtx(refuse_clusters=True)
    t, rep = tuning.autotune(ctx, None, "k", "g", cache=None, timer=lambda: 1.0)
    assert t["small_points"] == 0
    assert rep["tried"] == sum(len(choices) - 1 for _, choices in tuning.STAGES)  # one refused
    path = str(tmp_path / "old.json")
    json.dump({"g|k": {"tuning": {"spec_points": [0, 0, 0], "chunk_min": 128, "small_points": 0}}},
              open(path, "w"))
    ctx2 = FakeCtx()
    t2, rep2 = tuning.autotune(ctx2, None, "k", "g", cache=path)
    assert rep2["cached"] and t2["table_log2"] == 1 and t2["pass_shape"] == 0 and ctx2.t["chunk_min"] == 128


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
