"""Host logic of the launch-shape autotuner: workload keys, the JSON cache and
the choice, with a fake timer (no GPU)."""
import json

import pytest

from paper_2310_10642_gb300 import autotune as A


def _views(*sizes):
    return [dict(width=w, height=h) for w, h in sizes]


def test_workload_key_depends_on_what_timing_depends_on():
    v = _views((1352, 1014), (676, 507), (1352, 1014))
    k = A.workload_key("GB300", 1_000_000, v, 3, 2, 1, True)
    assert k == A.workload_key("GB300", 1_004_000, list(reversed(v)), 3, 2, 1, True)  # order, 2 digits of n
    assert "1352x1014*2" in k and "676x507*1" in k
    others = [A.workload_key("B200", 1_000_000, v, 3, 2, 1, True),
              A.workload_key("GB300", 2_000_000, v, 3, 2, 1, True),
              A.workload_key("GB300", 1_000_000, v[:2], 3, 2, 1, True),
              A.workload_key("GB300", 1_000_000, v, 1, 2, 1, True),
              A.workload_key("GB300", 1_000_000, v, 3, 2, 0, True),
              A.workload_key("GB300", 1_000_000, v, 3, 2, 1, False)]
    assert len({k, *others}) == 7


def test_select_fastest_and_ties():
    c = A.candidates((16, 32), (64, 256), (1,))
    assert len(c) == 4 and all(set(x) == set(A.KNOBS) for x in c)
    assert A.select([(c[0], 3.0), (c[1], 1.0), (c[2], 2.0)]) == c[1]
    assert A.select([(c[0], 1.0), (c[1], 1.0)]) == c[0]
    with pytest.raises(ValueError):
        A.select([])


def test_tune_with_times_once_then_reads_the_cache(tmp_path):
    path = str(tmp_path / "tune.json")
    cands = A.candidates((16, 32), (128, 256), (1,))
    ms = {(16, 128): 5.0, (16, 256): 4.0, (32, 128): 3.5, (32, 256): 3.9}
    calls = []

    def timer(c):
        calls.append(c)
        return ms[(c["tile_size"], c["batch_depth"])]

    choice, table = A.tune_with(timer, cands, "key1", path)
    assert choice == dict(tile_size=32, bin_size=32, batch_depth=128) and len(calls) == 4 and len(table) == 4
    stored = json.load(open(path))
    assert stored["key1"]["choice"] == choice

    def no_timer(c):
        raise AssertionError("cached workload re-timed")

    assert A.tune_with(no_timer, cands, "key1", path)[0] == choice
    # another workload is timed afresh and both entries are kept
    A.tune_with(lambda c: 1.0, cands, "key2", path)
    assert set(json.load(open(path))) == {"key1", "key2"}
    # no cache: always timed
    calls.clear()
    A.tune_with(timer, cands, "key1", None)
    assert len(calls) == 4


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    choice, _ = A.tune_with(lambda c: float(c["batch_depth"]), A.candidates((32,), (64, 128), (1,)), "k", str(path))
    assert choice == dict(tile_size=32, bin_size=32, batch_depth=64)


def test_candidates_pair_each_tile_with_the_bins_that_hold_it():
    c = A.candidates()
    pairs = sorted({(x["tile_size"], x["bin_size"]) for x in c})
    assert pairs == [(16, 16), (16, 32), (16, 64), (32, 32), (32, 64)]
    assert len(c) == len(pairs) * len(A.BATCH_DEPTHS)
    assert all(x["bin_size"] % x["tile_size"] == 0 and x["bin_size"] <= A.MAX_BIN for x in c)


def test_cache_entry_without_a_knob_is_timed_again(tmp_path):
    path = str(tmp_path / "tune.json")
    json.dump({"k": {"choice": {"tile_size": 32, "batch_depth": 256}, "table": []}}, open(path, "w"))
    calls = []
    choice, _ = A.tune_with(lambda c: calls.append(c) or float(c["bin_size"]), A.candidates((32,), (256,)), "k", path)
    assert len(calls) == 2 and choice == dict(tile_size=32, bin_size=32, batch_depth=256)
