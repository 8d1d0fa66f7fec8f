"""Host logic of the batched path's autotune cache (no GPU): shape classes,
the JSON file, and the hit/miss protocol with the tuner and the config setter
replaced by recording fakes."""
import json
import os

import pytest

import paper_2605_10390_gb300.tune_cache as tc

DEV = tc.device_key("GPU-X", 152, 10, 3)


def test_size_class_boundaries():
    # on-chip classes hold up to 1024 / 2048 / 4096 keys; 4097 is a large segment
    got = tc.batch_class([1024, 1025, 2048, 2049, 4096, 4097, 0], 32, True)
    assert got == "k32,v1,p32,s1024:1,s2048:2,s4096:2,sbig:1,n:16384"  # 14,339 keys


def test_counts_and_total_round_up_to_powers_of_two():
    a = tc.batch_class([100] * 5 + [10**6] * 3, 32, True, 32)
    b = tc.batch_class([900] * 8 + [600000] * 4, 32, True, 32)
    assert a == b  # 5 -> 8 and 3 -> 4 segments; both totals round up to 2^22
    assert tc.batch_class([100] * 9, 32, True) != tc.batch_class([100] * 8, 32, True)


def test_class_ignores_order_and_empty_segments_but_not_widths():
    sizes = [7, 3000, 50000, 1024]
    assert tc.batch_class(sizes, 64, False) == tc.batch_class(sizes[::-1] + [0, 0], 64, False)
    variants = {tc.batch_class(sizes, 64, False), tc.batch_class(sizes, 32, False),
                tc.batch_class(sizes, 64, True), tc.batch_class(sizes, 64, False, 24)}
    assert len(variants) == 4
    with pytest.raises(ValueError):
        tc.batch_class([-1], 32, True)


def test_round_trip_and_atomic_file(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = tc.TuneCache(path)
    assert c.get(DEV, "k32") is None
    c.put(DEV, "k32", {"small_capacity": 2048, "small_ctas_per_sm": 3, "large_form": 1, "digit_bits": 8}, 1.25)
    c.put(DEV, "k16", {"small_capacity": 0, "small_ctas_per_sm": 1, "large_form": 0, "digit_bits": 8})
    again = tc.TuneCache(path)
    assert again.get(DEV, "k32") == {"small_capacity": 2048, "small_ctas_per_sm": 3, "large_form": 1, "digit_bits": 8}
    assert again.get(DEV, "k16") == {"small_capacity": 0, "small_ctas_per_sm": 1, "large_form": 0, "digit_bits": 8}
    assert again.get("other-device", "k32") is None
    assert os.listdir(tmp_path / "sub") == ["tune.json"]  # no temporary file left behind
    d = json.load(open(path))
    assert d["version"] == tc.VERSION and d["entries"][f"{DEV}|k32"]["ms"] == 1.25


@pytest.mark.parametrize("bad", [
    {"small_capacity": 3000, "small_ctas_per_sm": 1, "large_form": 1, "digit_bits": 8},
    {"small_capacity": 1024, "small_ctas_per_sm": 0, "large_form": 1, "digit_bits": 8},
    {"small_capacity": 1024, "small_ctas_per_sm": 9, "large_form": 1, "digit_bits": 8},
    {"small_capacity": True, "small_ctas_per_sm": 1, "large_form": 1, "digit_bits": 8},
    {"small_capacity": 1024, "small_ctas_per_sm": 1, "large_form": 2, "digit_bits": 8},
    {"small_capacity": 1024, "small_ctas_per_sm": 1, "large_form": 1},
    {"small_capacity": 1024, "small_ctas_per_sm": 1, "large_form": 1, "digit_bits": 5},
    {"small_capacity": 1024, "small_ctas_per_sm": 1, "large_form": 1, "digit_bits": 9},
    {"small_capacity": 1024, "small_ctas_per_sm": 1},
    {"small_capacity": 1024},
    [1024, 2],
])
def test_invalid_entries_are_ignored_and_refused(tmp_path, bad):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"version": tc.VERSION, "entries": {
        f"{DEV}|bad": bad, f"{DEV}|good": {"small_capacity": 4096, "small_ctas_per_sm": 2, "large_form": 1, "digit_bits": 8}}}))
    c = tc.TuneCache(str(path))
    assert c.get(DEV, "bad") is None and c.get(DEV, "good") is not None
    if isinstance(bad, dict):
        with pytest.raises(ValueError):
            c.put(DEV, "bad", bad)


@pytest.mark.parametrize("text", ["", "{not json", "[]", '{"version": 0, "entries": {}}', '{"version": 1}'])
def test_unreadable_file_is_an_empty_cache(tmp_path, text):
    path = tmp_path / "tune.json"
    path.write_text(text)
    c = tc.TuneCache(str(path))
    assert c.entries == {}
    c.put(DEV, "x", {"small_capacity": 1024, "small_ctas_per_sm": 4, "large_form": 1, "digit_bits": 8})  # and is replaced on the next store
    assert tc.TuneCache(str(path)).get(DEV, "x") == {"small_capacity": 1024, "small_ctas_per_sm": 4, "large_form": 1, "digit_bits": 8}


def test_miss_tunes_and_stores_then_hit_only_sets(tmp_path, monkeypatch):
    calls = []

    def fake_tune(plan, segments, key_bits, precision_bits, stream):
        calls.append(("tune", plan, len(segments), key_bits, precision_bits))
        return {"small_capacity": 2048, "small_ctas_per_sm": 5, "large_form": 0, "digit_bits": 7}, 3.5

    def fake_set(plan, cap, ctas, form, width):
        calls.append(("set", plan, cap, ctas, form, width))

    monkeypatch.setattr(tc, "fsort_batch_autotune", fake_tune)
    monkeypatch.setattr(tc, "fsort_batch_set_config", fake_set)
    path = str(tmp_path / "tune.json")
    segs = [(0x1000, 0x2000, 3000), (0x3000, 0x4000, 70000)]
    cfg, ms, hit = tc.autotune_cached("plan-a", segs, 32, 32, has_values=True, path=path, device=DEV)
    assert (cfg, ms, hit) == ({"small_capacity": 2048, "small_ctas_per_sm": 5, "large_form": 0, "digit_bits": 7}, 3.5, False)
    assert calls == [("tune", "plan-a", 2, 32, 32)]
    # same shape class (another 3000-key and 70000-key segment pair): a hit, no timing
    segs2 = [(0x5000, 0x6000, 2500), (0x7000, 0x8000, 65000)]
    cfg, ms, hit = tc.autotune_cached("plan-b", segs2, 32, 32, has_values=True, path=path, device=DEV)
    assert (cfg, ms, hit) == ({"small_capacity": 2048, "small_ctas_per_sm": 5, "large_form": 0, "digit_bits": 7}, 3.5, True)
    assert calls[1:] == [("set", "plan-b", 2048, 5, 0, 7)]
    # another device or another class misses
    tc.autotune_cached("plan-c", segs2, 32, 32, has_values=True, path=path, device="GPU-Y/sm103/152sms")
    tc.autotune_cached("plan-d", segs2 * 3, 32, 32, has_values=True, path=path, device=DEV)
    assert [c[0] for c in calls[2:]] == ["tune", "tune"]


def test_segment_sizes_from_explicit_n_or_array_length():
    np = pytest.importorskip("numpy")
    assert tc.segment_sizes([(np.zeros(10, np.uint32), None), (0x10, None, 77)]) == [10, 77]
