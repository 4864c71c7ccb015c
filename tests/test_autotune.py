"""Decision logic of the autotuner (no GPU): nearest measured density, the
faster path wins, untuned classes fall back to packed, cache round trip."""
from paper_0712_0121_gb300.autotune import Tuner, _key


def table():
    return {_key(100, 200, "open", (31, 31)): {
        "density": [0.005, 0.05, 0.3], "packed_ms": [1.0, 1.0, 1.0], "rle_ms": [0.2, 0.9, 3.0],
        "band": 128}}


def test_choose_by_density(tmp_path):
    t = Tuner()
    t.table = table()
    assert t.choose(100, 200, "open", (31, 31), 0.004) == ("rle", 128)
    assert t.choose(100, 200, "open", (31, 31), 0.06) == ("rle", 128)
    assert t.choose(100, 200, "open", (31, 31), 0.25) == ("packed", 128)
    assert t.choose(5, 5, "open", (31, 31), 0.004, ref_size=(100, 200)) == ("rle", 128)
    assert t.choose(100, 200, "close", (3, 3), 0.01) == ("packed", 0)
    assert t.tuned(100, 200) and not t.tuned(5, 5)
    assert t.crossover(100, 200, "open", (31, 31)) == [0.005, 0.05]


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    t = Tuner(cache_path=p)
    t.table = table()
    t.save()
    assert Tuner(cache_path=p).table == table()


def test_word_tile_of_a_class():
    t = Tuner()
    t.table = table()
    assert t.words(100, 200, "open", (31, 31)) == 0          # older entries: the planner's choice
    t.table[_key(100, 200, "open", (31, 31))]["words"] = 4
    assert t.words(100, 200, "open", (31, 31)) == 4
    assert t.words(7, 7, "open", (31, 31), ref_size=(100, 200)) == 4
    assert t.words(100, 200, "close", (3, 3)) == 0            # untuned class


def _fake_tuner(band_ms, words_ms, rle_ms, seen):
    """A tuner whose timings come from tables instead of the GPU: packed
    batches cost band_ms[tile_rows] + words_ms[words_per_thread] per page-op,
    RLE batches rle_ms[density] per page-op; every timed batch is recorded."""
    t = Tuner(pages_per_class=3, reps=1, min_pixels=1)

    def time_batch(jobs, reps):
        seen.append(jobs)
        j = jobs[0]
        assert len({id(q["dst"]) for q in jobs}) == len(jobs)    # every job its own output
        if j["path"] == "rle":
            return rle_ms[j["src"][0]] * len(jobs)
        return (band_ms[j["tile_rows"]] + words_ms[j.get("words_per_thread", 0)]) * len(jobs)

    t._time_batch = time_batch
    return t


def test_tune_class_keeps_the_fastest_band_and_word_tile():
    seen = []
    t = _fake_tuner({32: 3.0, 64: 2.0, 128: 1.5, 256: 1.7}, {0: 0.0, 2: -0.25, 4: 0.5},
                    {0.005: 0.5, 0.05: 2.0}, seen)
    pages = {d: [(d, k) for k in range(3)] for d in (0.005, 0.05)}
    mid = [(0.08, k) for k in range(3)]
    outs = [object() for _ in range(3)]
    e = t.tune_class(100, 200, "open", (7, 7), densities=(0.005, 0.05), bands=(32, 64, 128, 256),
                     pages=pages, mid=mid, outs=outs)
    assert e["band"] == 128 and e["words"] == 2
    assert e["density"] == [0.005, 0.05]
    assert e["packed_ms"] == [1.25, 1.25] and e["rle_ms"] == [0.5, 2.0]   # per page-op
    # the density sweep times the packed path with the chosen band and word tile
    sweep = [b for b in seen if b[0]["src"][0] in (0.005, 0.05) and b[0]["path"] == "packed"]
    assert len(sweep) == 2
    assert all(q["tile_rows"] == 128 and q["words_per_thread"] == 2 for b in sweep for q in b)
    assert t.choose(100, 200, "open", (7, 7), 0.004) == ("rle", 128)
    assert t.choose(100, 200, "open", (7, 7), 0.06) == ("packed", 128)
    assert t.words(100, 200, "open", (7, 7)) == 2


def test_tune_class_keeps_the_planners_word_tile_unless_one_is_faster():
    seen = []
    t = _fake_tuner({64: 1.0, 128: 1.2}, {0: 0.0, 2: 0.1, 4: 0.0}, {0.02: 5.0}, seen)
    e = t.tune_class(100, 200, "erode", (3, 3), densities=(0.02,), bands=(64, 128),
                     pages={0.02: [(0.02, k) for k in range(3)]}, mid=[(0.08, k) for k in range(3)],
                     outs=[object() for _ in range(3)])
    assert e["band"] == 64 and e["words"] == 0          # a tie keeps the planner's choice
    assert t.crossover(100, 200, "erode", (3, 3)) == []
    assert t.choose(100, 200, "erode", (3, 3), 0.02) == ("packed", 64)
