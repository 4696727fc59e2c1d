"""Autotuner logic (no GPU): coordinate search and the JSON cache."""
import json

from paper_2006_14952_gb300 import autotune as A


def test_coordinate_search_finds_the_best_of_each_knob():
    # separable cost: each phase depends on its own knobs only
    best_want = {"tile_p2p_stage": 128, "tile_p2p_blocks": 4, "tile_m2l_blocks": 8, "tile_trav_blocks": 3}
    calls = []

    def measure(t):
        calls.append(dict(t))
        p2p = abs(t["tile_p2p_stage"] - 128) + 10 * abs(t["tile_p2p_blocks"] - 4)
        return {"t_p2p": 1.0 + p2p, "t_m2l": 1.0 + abs(t["tile_m2l_blocks"] - 8),
                "t_traverse": 1.0 + abs(t["tile_trav_blocks"] - 3)}

    best, trials = A.coordinate_search(measure)
    assert best == best_want
    assert len(calls) == sum(len(v[0]) for v in A.KNOBS.values())
    assert set(trials) == set(A.KNOBS)


def test_ties_keep_the_default():
    best, _ = A.coordinate_search(lambda t: {"t_p2p": 1.0, "t_m2l": 1.0, "t_traverse": 1.0})
    assert best == {k: v[0][0] for k, v in A.KNOBS.items()}


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "cache.json")
    k1 = A.cache_key("GB300", "nfw-2m", {"theta": 0.3, "order": 5})
    k2 = A.cache_key("GB300", "nfw-2m", {"theta": 0.3, "order": 6})
    assert k1 != k2
    assert A.lookup(path, k1) is None
    A.save(path, k1, {"tile_p2p_stage": 128}, {"tile_p2p_stage": {128: 1.0, 256: 2.0}})
    A.save(path, k2, {"tile_p2p_stage": 256}, {})
    assert A.lookup(path, k1) == {"tile_p2p_stage": 128}
    assert A.lookup(path, k2) == {"tile_p2p_stage": 256}
    data = json.load(open(path))
    assert data[k1]["trials_ms"]["tile_p2p_stage"]["128"] == 1.0
