"""Host logic of the autotuner (choice, size buckets, cache); no GPU."""
from paper_1512_03126_gb300 import autotune as A


def test_pick_takes_the_fastest_and_skips_missing():
    rs = [{"k": 1, "ms": 3.0}, {"k": 2, "ms": None}, {"k": 3, "ms": 1.5}, {"k": 4, "ms": 1.5}]
    assert A.pick(rs)["k"] == 3
    assert A.pick([{"ms": None}]) is None


def test_buckets_separate_sizes_species_and_reactions():
    assert A.bucket(3072, 1, 0) == "T2^12-S1-R0"
    assert A.bucket(3073, 1, 0) == "T2^12-S1-R0" != A.bucket(4097, 1, 0)
    assert A.bucket(2_400_000, 8, 14) == "T2^22-S8-R1"
    assert A.bucket(48_000, 3, 3) != A.bucket(48_000, 3, 0)


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("RDSPLIT_TUNE_CACHE", str(tmp_path / "sub" / "tune.json"))
    assert A.cache_get("x") is None
    A.cache_put("x", {"best": {"cluster": 2}})
    A.cache_put("y", {"best": {"mode": 1, "block": 128}})
    assert A.cache_get("x") == {"best": {"cluster": 2}}
    assert A.cache_get("y")["best"]["block"] == 128
