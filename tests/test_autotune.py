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
