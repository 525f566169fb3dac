"""Autotuner host logic on CPU: cache keys, the JSON cache and the choice,
with a fake timer in place of the GPU."""
import json

import pytest

from paper_1507_02525_gb300 import autotune


def test_cache_key_ignores_length_order_and_separates_configs():
    k1 = autotune.cache_key("GB300", False, 3, [8, 16, 32])
    k2 = autotune.cache_key("GB300", False, 3, [32, 8, 16])
    assert k1 == k2
    assert k1 != autotune.cache_key("GB300", True, 3, [8, 16, 32])
    assert k1 != autotune.cache_key("GB300", False, 3, [8, 16, 64])
    assert k1 != autotune.cache_key("other", False, 3, [8, 16, 32])


def test_pick_fastest_then_larger_segment():
    assert autotune.pick({(20, 4): 2.0, (23, 2): 1.5, (22, 4): 1.7}) == (23, 2)
    assert autotune.pick({(22, 4): 1.0, (23, 4): 1.0}) == (23, 4)
    with pytest.raises(ValueError):
        autotune.pick({})


def test_tune_times_once_then_reads_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    calls = []

    def timer(s, k):
        calls.append((s, k))
        return abs(s - 22) + 0.1 * k

    best = autotune.tune([1 << 24], 1, timer=timer, candidates=[(20, 4), (22, 2), (22, 4), (24, 2)])
    assert best == (22, 2)
    assert len(calls) == 4
    data = json.loads((tmp_path / "tune.json").read_text())
    (entry,) = data.values()
    assert entry["seg_log"] == 22 and entry["streams"] == 2 and len(entry["ms"]) == 4
    calls.clear()
    assert autotune.tune([1 << 24], 1, timer=timer) == (22, 2)
    assert calls == []  # served from the cache


def test_tune_drops_equivalent_large_segments(tmp_path, monkeypatch):
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    seen = []
    autotune.tune([1 << 16] * 4, 4, timer=lambda s, k: seen.append((s, k)) or 1.0,
                  candidates=[(20, 4), (22, 4), (23, 2), (16, 2)])
    # 4 signals of 2^16 (2^18 samples): segments of 2^20, 2^22, 2^23 all hold the whole batch
    assert (16, 2) in seen and sum(1 for s, _ in seen if s > 16) == 1


def test_tune_keeps_segment_sizes_that_group_signals(tmp_path, monkeypatch):
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    seen = []
    autotune.tune([1 << 16], 256, timer=lambda s, k: seen.append((s, k)) or 1.0,
                  candidates=[(20, 4), (22, 4), (23, 2), (24, 2), (26, 1)])
    # 256 signals of 2^16 (2^24 samples): 2^20, 2^22, 2^23 group 16, 64, 128 signals per
    # segment; 2^24 and 2^26 both hold the whole batch
    assert seen == [(20, 4), (22, 4), (23, 2), (24, 2)]


def test_corrupt_cache_is_ignored(tmp_path, monkeypatch):
    p = tmp_path / "tune.json"
    p.write_text("{not json")
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(p))
    assert autotune.load_cache() == {}
    assert autotune.tune([256], 1, timer=lambda s, k: float(s), candidates=[(12, 1), (13, 2)]) in [(12, 1), (13, 2)]


def test_objective_is_part_of_the_key(tmp_path, monkeypatch):
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    fwd = autotune.tune([1 << 24], 1, timer=lambda s, k: abs(s - 22) + 0.1 * k, objective="forward",
                        candidates=[(22, 2), (23, 2)])
    adj = autotune.tune([1 << 24], 1, timer=lambda s, k: abs(s - 23) + 0.1 * k, objective="adjoint",
                        candidates=[(22, 2), (23, 2)])
    both = autotune.tune([1 << 24], 1, timer=lambda s, k: float(k), candidates=[(22, 4), (23, 2)])
    assert (fwd, adj, both) == ((22, 2), (23, 2), (23, 2))
    assert len(json.loads((tmp_path / "tune.json").read_text())) == 3
    # adjoint=False is the forward objective, served from the cache
    assert autotune.tune([1 << 24], 1, timer=lambda s, k: 1 / 0, adjoint=False) == (22, 2)
    with pytest.raises(ValueError):
        autotune.tune([1 << 24], 1, timer=lambda s, k: 1.0, objective="sideways")


def test_tune_plan_searches_kernel_variants(tmp_path, monkeypatch):
    """Shape first, then each kernel variant in turn on the best shape; a
    variant is kept only when clearly faster; the choice is cached per
    objective under its own key."""
    monkeypatch.setenv("MRDFT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    seen = []

    def timer(o):
        seen.append(dict(o))
        ms = abs(o["seg_log"] - 21) + 0.1 * o["streams"] + 5.0
        ms -= 0.5 if o.get("fwd_cb") == 10 else 0.0       # clearly faster: kept
        ms -= 0.001 if o.get("dual_cols") is False else 0.0  # within the margin: not kept
        ms -= 0.3 if o.get("fwd_tree") is True else 0.0
        return ms

    best = autotune.tune_plan([1 << 24], 1, objective="forward", timer=timer,
                              candidates=[(20, 4), (21, 2), (22, 4)])
    assert best == {"seg_log": 21, "streams": 2, "tile_first": True, "fwd_cb": 10, "fwd_tree": True}
    names = {k for o in seen for k in o}
    assert {"fwd_cb", "fwd_rows_prefetch", "dual_cols", "fwd_tree", "tile_first"} <= names
    # the shape is searched with the in-tile levels both as one launch and per segment
    assert {(o["seg_log"], o.get("tile_first")) for o in seen} >= {(20, True), (20, False), (22, False)}
    assert not any("adj_cb" in o for o in seen)
    n = len(seen)
    assert autotune.tune_plan([1 << 24], 1, objective="forward", timer=lambda o: 1 / 0) == best
    assert len(seen) == n  # cached
    adj = autotune.tune_plan([1 << 24], 1, objective="adjoint",
                             timer=lambda o: float(o.get("adj_cb", 10)) - (0.5 if o.get("tile_first") is False else 0),
                             candidates=[(21, 2)])
    assert adj == {"seg_log": 21, "streams": 2, "tile_first": False, "adj_cb": 9}
    data = json.loads((tmp_path / "tune.json").read_text())
    assert sum(1 for k in data if k.endswith("|forward|opts")) == 1
    assert sum(1 for k in data if k.endswith("|adjoint|opts")) == 1


def test_knobs_only_where_they_change_the_plan():
    # no two-pass levels: nothing to tune beyond the shape
    assert autotune.knobs_for("forward", [1 << 14] * 8, 23) == ()
    # two-pass levels, but every signal fits in a segment: no tree switch
    names = [k for k, _ in autotune.knobs_for("forward", [1 << 18] * 64, 23)]
    assert "fwd_tree" not in names and "fwd_cb" in names
    assert "fwd_tree" in [k for k, _ in autotune.knobs_for("forward", [1 << 24], 21)]
    both = [k for k, _ in autotune.knobs_for("both", [1 << 24], 21)]
    assert both.count("dual_cols") == 1 and "adj_cb" in both and "fwd_cb" in both
