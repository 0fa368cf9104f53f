"""Continuous-batching server over the batched engine.

Requests (one simulation each: mesh, chemistry, initial counts, t_end, seed)
arrive over time.  The server admits them in arrival order while a device
memory budget and a slot limit allow, keeps their counts and period indices
resident on the device, and advances every admitted simulation by a time
slice of periods per engine launch; simulations that arrive while others run
join at the next slice, finished ones leave and free their memory.  A
request's latency is its completion time minus its arrival time (queueing,
upload, simulation and read-back included).

Large requests (n_tets * n_species at or above `dense_threshold`) do better
with the whole GPU than with one engine cluster: they go to a dense lane, a
worker thread that runs them one after another with rdsplit_run on its own
CUDA stream, overlapping the engine's launches on the other stream.

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
                 dense_stream=None):
        from . import rdsplit as rd
        self.rd = rd
        self.dense_threshold = float(dense_threshold)
        self.dense_stream = dense_stream
        self.budget = float(budget_bytes)
        self.max_slots = int(max_slots)
        self.slice = int(slice_periods)
        self.keep_counts = keep_counts
        self.engine = rd.rdsplit_engine_create(self.max_slots, 2**31 - 1)
        if stream is not None:
            rd.rdsplit_engine_set_stream(self.engine, stream)
        self.stream = stream
        self.used = 0
        self.active = {}

    def close(self):
        if self.engine is not None:
            self.rd.rdsplit_engine_destroy(self.engine)
            self.engine = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _admit(self, req, now: float, rec: Record):
        w = req.workload() if callable(getattr(req, "workload", None)) else req.workload
        nbytes = device_bytes(w.mesh.n_tets, w.model.n_species)
        sim = self.rd.Simulation(w.mesh, w.model, w.counts, stream=self.stream)
        slot = self.rd.rdsplit_engine_add(self.engine, sim.h, w.t_end, w.seed)
        tau = sim.tau
        t, P = 0.0, 0
        while t < w.t_end:
            t = w.t_end if t + tau > w.t_end else t + tau
            P += 1
        rec.admitted = now
        rec.tet_periods = w.mesh.n_tets * P
        self.active[slot] = (rec, sim, nbytes)
        self.used += nbytes

    def _dense_worker(self, jobs, done, lock, t0, clock):
        """Dense lane: run each large request alone, in arrival order."""
        rd = self.rd
        while True:
            item = jobs.get()
            if item is None:
                return
            rec, w = item
            rec.admitted = clock() - t0
            with rd.Simulation(w.mesh, w.model, w.counts, stream=self.dense_stream) as sim:
                tau = sim.tau
                t, P = 0.0, 0
                while t < w.t_end:
                    t = w.t_end if t + tau > w.t_end else t + tau
                    P += 1
                rec.tet_periods = w.mesh.n_tets * P
                sim.run(w.t_end, w.seed)
                counts = sim.counts()
            if self.keep_counts:
                rec.counts = counts
            rec.done = clock() - t0
            with lock:
                done.append(rec)

    def serve(self, requests, prepared=None, clock=time.perf_counter):
        """Serve `requests` (objects with .rid, .arrival in seconds from the
        start, and .workload); `prepared` may map rid -> Workload built ahead
        of time (inputs arriving with the request).  Returns the records in
        completion order."""
        rd = self.rd
        order = sorted(requests, key=lambda r: r.arrival)
        pending = deque(order)
        waiting = deque()
        records = {}
        done = []
        lock = threading.Lock()
        jobs = queue.Queue()
        t0 = clock()
        worker = None
        if self.dense_threshold < float("inf"):
            worker = threading.Thread(target=self._dense_worker, args=(jobs, done, lock, t0, clock), daemon=True)
            worker.start()
        while pending or waiting or self.active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                records[r.rid] = Record(r.rid, r.arrival)
                w = prepared[r.rid] if prepared is not None else r.workload()
                if w.mesh.n_tets * w.model.n_species >= self.dense_threshold:
                    jobs.put((records[r.rid], w))
                else:
                    waiting.append(r)
            while waiting and len(self.active) < self.max_slots:
                r = waiting[0]
                w = prepared[r.rid] if prepared is not None else r.workload()
                need = device_bytes(w.mesh.n_tets, w.model.n_species)
                if self.used + need > self.budget and self.active:
                    break
                waiting.popleft()
                self._admit(_Prepared(r.rid, w), clock() - t0, records[r.rid])
            if self.active:
                rd.rdsplit_engine_step(self.engine, self.slice)
                for slot in rd.rdsplit_engine_poll(self.engine):
                    rec, sim, nbytes = self.active.pop(slot)
                    counts = sim.counts()          # the result goes back to the host
                    if self.keep_counts:
                        rec.counts = counts
                    rec.done = clock() - t0
                    sim.close()
                    self.used -= nbytes
                    with lock:
                        done.append(rec)
            elif pending:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        if worker is not None:
            jobs.put(None)
            worker.join()
        return done


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
