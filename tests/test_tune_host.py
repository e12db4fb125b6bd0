"""Host logic of the launch-shape autotuner (no GPU: a fake timer)."""
import json

from paper_1310_1854_gb300 import tune


def test_search_picks_smallest_median():
    calls = []

    def fake(shape):
        calls.append(shape)
        lanes, block, _ = shape
        return {1: 3.0, 2: 2.0, 4: 5.0}[lanes] + block / 1000.0

    best, table = tune.search(((1, 128, 0), (2, 128, 0), (2, 256, 0), (4, 128, 0)), fake, repeats=3)
    assert best == (2, 128, 0)
    assert len(calls) == 12
    assert table["2,128,0"] == 2.128


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    k = tune.shape_key("NVIDIA GB300", "fp32", 100_000, 1_000_000)
    assert k == "NVIDIA GB300|fp32|M2^17|N2^20"
    assert tune.load_cache(p) == {}
    tune.store(k, {"lanes_per_ray": 1, "block": 256, "blocks_per_sm": 0}, p)
    tune.store("other", {"lanes_per_ray": 4, "block": 128, "blocks_per_sm": 0}, p)
    d = tune.load_cache(p)
    assert d[k]["lanes_per_ray"] == 1 and d["other"]["block"] == 128
    with open(p, "w") as f:
        f.write("{broken")
    assert tune.load_cache(p) == {}
    json.dumps(d)
