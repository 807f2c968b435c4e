"""Host logic of the autotuner's table (no GPU): keys, lookup fallbacks and
shape tuples; and the committed table's entries are well formed."""
import numpy as np

from paper_1504_00353_gb300 import autotune, synth


def test_keys_and_lookup_fallback():
    m = synth.frozen_mask(1024, 512, 2.5)
    other = synth.frozen_mask(1024, 512, 3.0)
    table = {"GPU X": {
        autotune.code_key(1024, 512, m, "i8"): {"threads": 32, "tag": "exact"},
        autotune.code_key(1024, 512, other, "i8"): {"threads": 64, "tag": "other mask"},
        autotune.code_key(1024, 512, m, "i8", latency=True): {"threads": 256, "tag": "latency"},
        "mixed_i8": {"threads": 32},
    }}
    assert autotune.lookup(1024, 512, m, "i8", table, "GPU X")["tag"] == "exact"
    assert autotune.lookup(1024, 512, m, "i8", table, "GPU X", latency=True)["tag"] == "latency"
    # another mask of the same (N, K, dtype) is the fallback; other devices see nothing
    m2 = synth.frozen_mask(1024, 512, 1.0)
    assert autotune.lookup(1024, 512, m2, "i8", table, "GPU X")["threads"] in (32, 64)
    assert autotune.lookup(1024, 512, m, "f32", table, "GPU X") is None
    assert autotune.lookup(1024, 512, m, "i8", table, "GPU Y") is None
    assert autotune.lookup(2048, 512, m, "i8", table, "GPU X") is None


def test_shape_tuple_roundtrip():
    s = dict(threads=128, smem_stage_max=2048, warp_stage_max=1024, ctas_per_sm=8,
             stage_channel=1, reg_subtree=512, frames_per_cta=1, local_leaves=1,
             compile_form="subtrees")
    assert autotune._shape(autotune._shape_key(s)) == s
    # defaults fill missing keys
    k = autotune._shape_key(dict(threads=32, smem_stage_max=256, warp_stage_max=2048))
    assert autotune._shape(k)["stage_channel"] == 2 and autotune._shape(k)["reg_subtree"] == 256
    assert autotune._shape(k)["frames_per_cta"] == 1 and autotune._shape(k)["local_leaves"] == 0


def test_mask_hash_is_stable_and_distinguishes():
    a = synth.frozen_mask(256, 128, 3.0)
    assert autotune.mask_hash(a) == autotune.mask_hash(a.copy())
    b = a.copy()
    b[np.flatnonzero(a == 0)[0]] = 1
    assert autotune.mask_hash(a) != autotune.mask_hash(b)


def test_committed_table_is_well_formed():
    t = autotune.load_table()
    assert t, "tuned_shapes.json is missing"
    for dev, entries in t.items():
        for key, e in entries.items():
            if key.startswith("mixed_"):
                assert e["threads"] % 32 == 0 and len(e["smem_stage_max"]) == len(e["warp_stage_max"])
                continue
            parts = key.split("_")
            assert parts[3] in ("f32", "i8") and int(parts[0]) >= int(parts[1])
            assert e["threads"] % 32 == 0 and e["threads"] <= 1024
            assert ("latency_us" in e) == key.endswith("_lat")


def test_module_entry_point_defines_everything_it_uses():
    """Run as a script (python -m ...), main() must come after every module-level
    definition the tuning path uses: the main guard is the last statement."""
    import ast
    tree = ast.parse(open(autotune.__file__).read())
    last = tree.body[-1]
    assert isinstance(last, ast.If) and "__main__" in ast.dump(last.test)
    assert autotune.SHAPE_DEFAULTS["compile_form"] in autotune.COMPILE_FORM


def test_throughput_search_reaches_form_and_register_subtree():
    """The coordinate search (threads, stage cap, warp threshold, resident CTAs,
    frames per CTA, compile form, register-subtree size) run against a synthetic
    cost table with no GPU: it must end at the cheapest shape when each knob's
    best value can be found one coordinate at a time."""
    class FakeTuner(autotune.CodeTuner):
        def __init__(self):  # no device: only the search logic
            self.N, self.K, self.dtype, self.latency = 32768, 29492, "i8", False
            self.seen, self.log, self.asked = {}, None, []

        def measure(self, shapes):
            for s in map(self.clamp, shapes):
                self.asked.append(s)
                t = 10.0
                t -= {32: 2.0, 64: 1.0}.get(s["threads"], 0.0)
                t -= {1024: 1.0}.get(s["smem_stage_max"], 0.0)
                t -= {4: 1.5, 2: 0.5}.get(s["frames_per_cta"], 0.0)
                t -= 0.8 if s["compile_form"] == "subtrees" else 0.0
                t -= 0.4 if s["reg_subtree"] == 512 else 0.0
                self.seen[autotune._shape_key(s)] = t

    t = FakeTuner()
    best, cost = t.tune()
    assert best["threads"] == 32 and best["frames_per_cta"] == 4
    assert best["smem_stage_max"] == 1024
    assert best["compile_form"] == "subtrees" and best["reg_subtree"] == 512
    assert cost == min(t.seen.values())
    assert any(s["reg_subtree"] == 512 for s in t.asked)
