"""Host logic of the continuous-batching server (admission by budget and
slots, arrival order, completion bookkeeping) against a fake engine; no GPU."""
import types

import numpy as np

from paper_1512_03126_gb300 import serving as SV


class FakeRd:
    """Stands in for the C-ABI binding: each simulation finishes after a
    fixed number of engine steps."""

    def __init__(self, steps_to_finish):
        self.steps_to_finish = steps_to_finish
        self.slots = {}
        self.finished = []
        self.max_active = 0
        self.admitted_order = []

    def rdsplit_engine_create(self, max_slots, cap):
        return "engine"

    def rdsplit_engine_destroy(self, e):
        pass

    def rdsplit_engine_add(self, e, h, t_end, seed):
        slot = next(s for s in range(1000) if s not in self.slots)
        self.slots[slot] = self.steps_to_finish
        self.max_active = max(self.max_active, len(self.slots))
        self.admitted_order.append(h.rid)
        return slot

    def rdsplit_engine_step(self, e, n):
        for s in list(self.slots):
            self.slots[s] -= 1
            if self.slots[s] == 0:
                del self.slots[s]
                self.finished.append(s)

    def rdsplit_engine_poll(self, e, max_slots=4096):
        out, self.finished = self.finished, []
        return out

    class Simulation:
        def __init__(self, mesh, model, counts, stream=None):
            self.h = types.SimpleNamespace(rid=mesh.rid)
            self.tau = 1e-3

        def counts(self):
            return np.zeros(1)

        def close(self):
            pass


def _req(rid, arrival, T=100, S=1):
    mesh = types.SimpleNamespace(n_tets=T, rid=rid)
    model = types.SimpleNamespace(n_species=S)
    w = types.SimpleNamespace(mesh=mesh, model=model, counts=None, t_end=0.01, seed=rid)
    return types.SimpleNamespace(rid=rid, arrival=arrival), w


def _server(fake, **kw):
    srv = SV.Server.__new__(SV.Server)
    srv.rd = fake
    srv.budget = kw.get("budget", 1e18)
    srv.max_slots = kw.get("slots", 2)
    srv.slice = 1
    srv.keep_counts = False
    srv.engine = "engine"
    srv.stream = None
    srv.used = 0
    srv.active = {}
    srv.dense_threshold = float("inf")
    srv.dense_lanes = kw.get("lanes", 1)
    srv.dense_streams = [None] * srv.dense_lanes
    srv._lock = SV.threading.Lock()
    srv.host_s = {"admit": 0.0, "step": 0.0, "retire": 0.0}
    return srv


def test_slot_limit_and_fifo_admission():
    fake = FakeRd(steps_to_finish=3)
    fake.Simulation = FakeRd.Simulation
    pairs = [_req(i, 0.0) for i in range(5)]
    srv = _server(fake, slots=2)
    recs = srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert fake.max_active == 2
    assert fake.admitted_order == [0, 1, 2, 3, 4]
    assert sorted(r.rid for r in recs) == [0, 1, 2, 3, 4]
    assert srv.used == 0 and not srv.active


def test_memory_budget_limits_admission():
    fake = FakeRd(steps_to_finish=2)
    fake.Simulation = FakeRd.Simulation
    pairs = [_req(i, 0.0, T=1000) for i in range(4)]
    one = SV.device_bytes(1000, 1)
    srv = _server(fake, slots=10, budget=2.5 * one)
    srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert fake.max_active == 2


def test_latency_includes_queueing():
    fake = FakeRd(steps_to_finish=1)
    fake.Simulation = FakeRd.Simulation
    clock = {"t": 0.0}

    def tick():
        clock["t"] += 0.001
        return clock["t"]

    pairs = [_req(i, 0.0) for i in range(3)]
    srv = _server(fake, slots=1)
    recs = srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs}, clock=tick)
    lat = {r.rid: r.latency for r in recs}
    assert lat[0] < lat[1] < lat[2]
    s = SV.summarize(recs)
    assert s["requests"] == 3 and s["p99_ms"] >= s["p50_ms"]


def test_dense_lane_takes_large_requests():
    fake = FakeRd(steps_to_finish=2)

    class Sim(FakeRd.Simulation):
        ran = []

        def run(self, t_end, seed):
            Sim.ran.append(self.h.rid)

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

    fake.Simulation = Sim
    small = [_req(i, 0.0, T=10) for i in range(3)]
    large = [_req(10 + i, 0.0, T=10_000) for i in range(2)]
    pairs = small + large
    srv = _server(fake, slots=4)
    srv.dense_threshold = 5_000
    recs = srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert sorted(Sim.ran) == [10, 11]
    assert sorted(fake.admitted_order) == [0, 1, 2]
    assert sorted(r.rid for r in recs) == [0, 1, 2, 10, 11]


class _DenseSim(FakeRd.Simulation):
    """A dense-lane simulation that records how many run at once."""
    lock = SV.threading.Lock()
    running = 0
    peak = 0
    fail_rid = None

    def run(self, t_end, seed):
        import time
        with _DenseSim.lock:
            _DenseSim.running += 1
            _DenseSim.peak = max(_DenseSim.peak, _DenseSim.running)
        time.sleep(0.02)
        with _DenseSim.lock:
            _DenseSim.running -= 1
        if self.h.rid == _DenseSim.fail_rid:
            raise RuntimeError("planted failure")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def _dense_setup(budget_units, lanes, fail_rid=None):
    fake = FakeRd(steps_to_finish=2)
    fake.Simulation = _DenseSim
    _DenseSim.running = _DenseSim.peak = 0
    _DenseSim.fail_rid = fail_rid
    pairs = [_req(i, 0.0, T=10_000) for i in range(4)]
    one = SV.device_bytes(10_000, 1)
    srv = _server(fake, slots=4, budget=budget_units * one, lanes=lanes)
    srv.dense_threshold = 5_000
    return srv, pairs


def test_dense_lanes_share_the_memory_budget():
    """Dense-lane requests reserve their device memory at admission: with room
    for one at a time, two lanes never run two at once; with room for all,
    both lanes overlap.  The budget is released when they finish."""
    srv, pairs = _dense_setup(1.5, lanes=2)
    recs = srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert sorted(r.rid for r in recs) == [0, 1, 2, 3]
    assert _DenseSim.peak == 1 and srv.used == 0
    srv, pairs = _dense_setup(10, lanes=2)
    srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert _DenseSim.peak == 2 and srv.used == 0


def test_dense_lane_error_is_raised():
    """A failure in a dense lane is raised from serve(), not dropped."""
    import pytest
    srv, pairs = _dense_setup(10, lanes=2, fail_rid=2)
    with pytest.raises(RuntimeError, match="request 2 failed"):
        srv.serve([p[0] for p in pairs], {p[0].rid: p[1] for p in pairs})
    assert srv.used == 0


def test_server_sets_the_engine_cluster_size(monkeypatch):
    from paper_1512_03126_gb300 import rdsplit as rd
    calls = []
    monkeypatch.setattr(rd, "rdsplit_engine_create", lambda n, cap: "eng")
    monkeypatch.setattr(rd, "rdsplit_engine_set_concurrency", lambda e, f, c: calls.append(("conc", e, f, c)))
    monkeypatch.setattr(rd, "rdsplit_engine_set_slice_work", lambda e, w: calls.append(("work", e, w)))
    monkeypatch.setattr(rd, "rdsplit_engine_destroy", lambda e: calls.append(("destroy", e)))
    srv = SV.Server(budget_bytes=1e9, max_slots=4, cluster=8, slice_work=1000)
    srv.close()
    assert calls == [("conc", "eng", 0, 8), ("work", "eng", 1000), ("destroy", "eng")]
    calls.clear()
    SV.Server(budget_bytes=1e9, max_slots=4).close()
    assert calls == [("conc", "eng", 0, 2), ("destroy", "eng")]
