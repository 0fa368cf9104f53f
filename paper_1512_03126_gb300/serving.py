"""Continuous-batching server over the batched engine.

Requests (one simulation each: mesh, chemistry, initial counts, t_end, seed)
arrive over time.  The server admits them in arrival order while a device
memory budget and a slot limit allow, keeps their counts and period indices
resident on the device, and advances every admitted simulation by a time
slice of periods per engine launch; simulations that arrive while others run
join at the next slice, finished ones leave and free their memory.  A
request's latency is its completion time minus its arrival time (queueing,
upload, simulation and read-back included).

Each simulation in the engine runs on a thread-block cluster of `cluster`
CTAs (1, 2, 4 or 8): larger clusters shorten the largest requests, which set
the span of a saturated mix.

With `slice_work` > 0 a launch advances a large simulation by fewer periods
(about slice_work / n_tets), so that the slices of one launch cost about
the same and no cluster idles behind the largest request.

Requests with n_tets * n_species at or above `dense_threshold` can instead
go to a dense lane: `dense_lanes` worker threads, each running its requests
one after another with rdsplit_run (every tet every period, the whole GPU)
on its own CUDA stream, overlapping the engine's launches and each other.
Their device memory counts against the same budget, reserved at admission
and released when they finish.

Each simulation's random streams are keyed by its own seed, period index and
canonical tet ids, so its result is the same whether it runs alone or mixed
with others, in either lane.  The host code here is argument marshalling and bookkeeping;
all simulation work runs in the library's kernels.
"""
from __future__ import annotations

import queue
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


def device_bytes(n_tets: int, n_species: int) -> int:
    """Device memory a simulation holds in the library (mesh, model state and
    the engine's per-simulation lists), used for admission."""
    per_tet = 16 + 32 + 8 + 8 + 4 + 8 + 8 + 8 + 32 + 8
    per_tet_species = 4 + 4 + 32 + 32 + 4
    return int(n_tets) * per_tet + int(n_tets) * int(n_species) * per_tet_species


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    tet_periods: int = 0
    counts: np.ndarray | None = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Server:
    """Admit, batch and advance simulations; see the module docstring."""

    def __init__(self, budget_bytes: float = 150e9, max_slots: int = 128, slice_periods: int = 256,
                 stream=None, keep_counts: bool = False, dense_threshold: float = float("inf"),
                 dense_stream=None, dense_lanes: int = 1, slice_work: int = 0, cluster: int = 2):
        from . import rdsplit as rd
        self.rd = rd
        self.dense_threshold = float(dense_threshold)
        self.dense_lanes = max(1, int(dense_lanes))
        # one CUDA stream per dense lane: the caller's dense_stream for the
        # first lane (None: the legacy default stream), new streams for the others
        self.dense_streams = [dense_stream]
        if self.dense_lanes > 1:
            import torch
            self.dense_streams += [torch.cuda.Stream() for _ in range(self.dense_lanes - 1)]
        self.budget = float(budget_bytes)
        self.max_slots = int(max_slots)
        self.slice = int(slice_periods)
        self.keep_counts = keep_counts
        self.engine = rd.rdsplit_engine_create(self.max_slots, 2**31 - 1)
        rd.rdsplit_engine_set_concurrency(self.engine, 0, int(cluster))
        if slice_work:
            rd.rdsplit_engine_set_slice_work(self.engine, int(slice_work))
        if stream is not None:
            rd.rdsplit_engine_set_stream(self.engine, stream)
        self.stream = stream
        self.used = 0              # device bytes held by admitted simulations (both lanes)
        self.active = {}
        self._lock = threading.Lock()
        self.host_s = {"admit": 0.0, "step": 0.0, "retire": 0.0}   # wall time of the serving loop by phase

    def close(self):
        if self.engine is not None:
            self.rd.rdsplit_engine_destroy(self.engine)
            self.engine = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _admit(self, rid: int, w, now: float, rec: Record, nbytes: int):
        sim = self.rd.Simulation(w.mesh, w.model, w.counts, stream=self.stream)
        try:
            slot = self.rd.rdsplit_engine_add(self.engine, sim.h, w.t_end, w.seed)
        except Exception:
            sim.close()
            raise
        rec.admitted = now
        rec.tet_periods = w.mesh.n_tets * _periods(sim.tau, w.t_end)
        self.active[slot] = (rec, sim, nbytes)

    def _dense_worker(self, lane: int, jobs, done, t0, clock, errors):
        """Dense lane: run each large request alone on this lane's stream, in
        the order the lanes take them; its device memory was reserved at
        admission and is released here."""
        rd = self.rd
        stream = self.dense_streams[lane]
        while True:
            item = jobs.get()
            if item is None:
                return
            rec, w, nbytes = item
            try:
                rec.admitted = clock() - t0
                with rd.Simulation(w.mesh, w.model, w.counts, stream=stream) as sim:
                    rec.tet_periods = w.mesh.n_tets * _periods(sim.tau, w.t_end)
                    sim.run(w.t_end, w.seed)
                    counts = sim.counts()
                if self.keep_counts:
                    rec.counts = counts
                rec.done = clock() - t0
                with self._lock:
                    done.append(rec)
            except BaseException as e:   # reported by serve(), never dropped
                with self._lock:
                    errors.append((rec.rid, e))
            finally:
                with self._lock:
                    self.used -= nbytes
                    self._dense_out -= 1

    def serve(self, requests, prepared=None, clock=time.perf_counter):
        """Serve `requests` (objects with .rid, .arrival in seconds from the
        start, and .workload); `prepared` may map rid -> Workload built ahead
        of time (inputs arriving with the request).  Returns the records in
        completion order.  Requests are admitted in arrival order while the
        device budget (both lanes) and the engine's slots allow; an error in
        either lane is raised here."""
        rd = self.rd
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        records = {}
        done = []
        errors = []
        jobs = queue.Queue()
        self._dense_out = 0
        t0 = clock()
        workers = []
        if self.dense_threshold < float("inf"):
            for lane in range(self.dense_lanes):
                th = threading.Thread(target=self._dense_worker, args=(lane, jobs, done, t0, clock, errors),
                                      daemon=True)
                th.start()
                workers.append(th)
        try:
            while pending or waiting or self.active or self._dense_out > 0:
                if errors:
                    rid, e = errors[0]
                    raise RuntimeError(f"request {rid} failed in the dense lane: {e}") from e
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    r = pending.popleft()
                    records[r.rid] = Record(r.rid, r.arrival)
                    waiting.append(r)
                while waiting:
                    r = waiting[0]
                    w = prepared[r.rid] if prepared is not None else r.workload()
                    need = device_bytes(w.mesh.n_tets, w.model.n_species)
                    dense = workers and w.mesh.n_tets * w.model.n_species >= self.dense_threshold
                    with self._lock:
                        busy = bool(self.active) or self._dense_out > 0
                        if self.used + need > self.budget and busy:
                            break
                        if not dense and len(self.active) >= self.max_slots:
                            break
                        self.used += need
                        if dense:
                            self._dense_out += 1
                    waiting.popleft()
                    if dense:
                        jobs.put((records[r.rid], w, need))
                    else:
                        ta = clock()
                        try:
                            self._admit(r.rid, w, clock() - t0, records[r.rid], need)
                        except Exception:
                            with self._lock:
                                self.used -= need
                            raise
                        self.host_s["admit"] += clock() - ta
                if self.active:
                    ts = clock()
                    rd.rdsplit_engine_step(self.engine, self.slice)
                    tr = clock()
                    self.host_s["step"] += tr - ts
                    for slot in rd.rdsplit_engine_poll(self.engine):
                        rec, sim, nbytes = self.active.pop(slot)
                        counts = sim.counts()          # the result goes back to the host
                        if self.keep_counts:
                            rec.counts = counts
                        rec.done = clock() - t0
                        sim.close()
                        with self._lock:
                            self.used -= nbytes
                            done.append(rec)
                    self.host_s["retire"] += clock() - tr
                else:
                    wait = pending[0].arrival - (clock() - t0) if pending else 0.001
                    if wait > 0:
                        time.sleep(min(wait, 0.002))
        finally:
            for _ in workers:
                jobs.put(None)
            for th in workers:
                th.join()
        if errors:
            rid, e = errors[0]
            raise RuntimeError(f"request {rid} failed in the dense lane: {e}") from e
        return done


def _periods(tau: float, t_end: float) -> int:
    """Periods of Algorithm 1 from 0 to t_end (the last one shortened)."""
    t, P = 0.0, 0
    while t < t_end:
        t = t_end if t + tau > t_end else t + tau
        P += 1
    return P


@dataclass
class _Prepared:
    rid: int
    workload: object


def summarize(records, wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in records]) * 1e3
    units = sum(r.tet_periods for r in records)
    span = wall if wall is not None else max(r.done for r in records) - min(r.arrival for r in records)
    return {"requests": len(records), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput": units / span if span > 0 else None, "tet_periods": units, "span_s": span}
