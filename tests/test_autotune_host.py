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


class _FakeEngineRd:
    """Stands in for the binding: records the cluster size of each engine and
    lets the timing stub report a cost per cluster size."""

    def __init__(self):
        self.cluster = {}
        self.launched = []
        self.destroyed = 0

    def rdsplit_get_shape(self, h):
        return (100, 1)

    def rdsplit_engine_create(self, n, cap):
        e = object()
        self.cluster[e] = None
        return e

    def rdsplit_engine_set_stream(self, e, s):
        pass

    def rdsplit_engine_set_concurrency(self, e, in_flight, cluster):
        assert in_flight == 0
        self.cluster[e] = cluster

    def rdsplit_engine_add(self, e, h, t_end, seed):
        pass

    def rdsplit_engine_step(self, e, n):
        self.launched.append(self.cluster[e])

    def rdsplit_engine_poll(self, e, n):
        return []

    def rdsplit_engine_schedule(self, e):
        c = self.cluster[e]
        return (152 // c, c, 152 // c)

    def rdsplit_engine_destroy(self, e):
        self.destroyed += 1


def test_tune_engine_times_every_cluster_size_and_keeps_the_fastest(tmp_path, monkeypatch):
    import types
    monkeypatch.setenv("RDSPLIT_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(A, "_device_name", lambda: "fake-gpu")
    cost = {1: 9.0, 2: 4.0, 4: 2.5, 8: 3.0}
    rd = _FakeEngineRd()

    def timed(fn, stream):
        fn()
        return cost[rd.launched[-1]]

    monkeypatch.setattr(A, "_timed", timed)
    resets = []
    sims = [types.SimpleNamespace(h=i) for i in range(3)]
    out = A.tune_engine(rd, sims, [0.1] * 3, [1, 2, 3], lambda: resets.append(1), None,
                        clusters=(2, 4, 8, 1), use_cache=True, shape_key="mix")
    assert rd.launched == [2, 4, 8, 1] and len(resets) == 4 and rd.destroyed == 4
    assert out["best"] == {"cluster": 4}
    assert [r["cluster"] for r in out["results"]] == [2, 4, 8, 1]
    assert out["results"][1]["in_flight"] == 38
    # a second call with the same shape key comes from the cache
    again = A.tune_engine(rd, sims, [0.1] * 3, [1, 2, 3], lambda: resets.append(1), None,
                          clusters=(2, 4, 8, 1), use_cache=True, shape_key="mix")
    assert again["cached"] and again["best"] == {"cluster": 4} and len(rd.launched) == 4
