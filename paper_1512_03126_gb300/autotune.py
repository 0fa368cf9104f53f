"""Autotuner of the launch shapes (none of them changes a result: every
draw is keyed by seed, period and canonical tet id, and every transfer is an
integer sum).

  engine       CTAs per simulation (1, 2, 4 or 8) of the batched engine, at the
               number of clusters that fit on the GPU at once
  period       the dense period kernel: one pass or two passes, and the
               block size
  single mesh  the dense period loop against the batched engine for one
               simulation

Each candidate is timed on the caller's own workload with CUDA events; the
choice is cached per (GPU name, kind, size bucket) in a JSON file
(RDSPLIT_TUNE_CACHE, default ~/.cache/rdsplit/tune.json) so that later runs
of the same shape reuse it.  The host code here only times library calls.
"""
from __future__ import annotations

import json
import math
import os
import threading

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("RDSPLIT_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rdsplit",
                                                             "tune.json"))


def bucket(n_tets: int, n_species: int, n_reactions: int) -> str:
    """Size class of a workload: tets by power of two, species, with or
    without reactions."""
    return f"T2^{max(0, math.ceil(math.log2(max(1, int(n_tets)))))}-S{int(n_species)}-R{int(n_reactions > 0)}"


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def cache_get(key: str):
    with _lock:
        try:
            return json.load(open(cache_path())).get(key)
        except (OSError, ValueError):
            return None


def cache_put(key: str, value) -> None:
    with _lock:
        path = cache_path()
        try:
            data = json.load(open(path))
        except (OSError, ValueError):
            data = {}
        data[key] = value
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass


def pick(results: list) -> dict:
    """The fastest candidate (ties: the first listed)."""
    best = None
    for r in results:
        if r.get("ms") is None:
            continue
        if best is None or r["ms"] < best["ms"]:
            best = r
    return best


def _timed(fn, stream) -> float:
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


DENSE_CANDIDATES = [(1, 32), (1, 64), (1, 128), (1, 256), (2, 64), (2, 256)]


def tune_period(rd, w, stream, periods: int = 48, candidates=None, use_cache: bool = True) -> dict:
    """Dense period kernel for workload w (mesh, model, counts, seed): time
    `periods` periods from the initial state per candidate (mode, block);
    also the batched engine on the same periods.  Returns {"best": {...},
    "results": [...]} with "best" the fastest dense form (the engine's time
    is reported for the single-mesh choice)."""
    key = f"{_device_name()}|period|{bucket(w.mesh.n_tets, w.model.n_species, w.model.n_reactions)}"
    if use_cache:
        hit = cache_get(key)
        if hit:
            return dict(hit, cached=True)
    import numpy as np
    import torch
    cands = candidates or DENSE_CANDIDATES
    results = []
    d_counts = torch.from_numpy(np.ascontiguousarray(w.counts, dtype=np.int32)).cuda()
    sim = rd.Simulation(w.mesh, w.model, stream=stream)
    try:
        tau = sim.tau
        n = max(1, min(int(periods), int(w.t_end / tau) if math.isfinite(tau) and tau > 0 else 1))

        def dense():
            rd.rdsplit_set_counts_device(sim.h, d_counts)
            rd.rdsplit_set_time(sim.h, 0.0, 0)
            sim.run_periods(n, w.seed)

        for mode, block in cands:
            rd.rdsplit_set_period_kernel(sim.h, mode, block)
            dense()                                   # warm
            ms = min(_timed(dense, stream) for _ in range(2))
            results.append({"form": "dense", "mode": mode, "block": block, "ms": ms, "periods": n})
        rd.rdsplit_set_period_kernel(sim.h, 0, 0)
        for cluster in (1, 2, 4, 8):
            ms = []
            for _ in range(3):
                eng = rd.rdsplit_engine_create(1, w.mesh.n_tets)
                try:
                    rd.rdsplit_engine_set_stream(eng, stream)
                    rd.rdsplit_engine_set_concurrency(eng, 0, cluster)

                    def batched():
                        rd.rdsplit_set_counts_device(sim.h, d_counts)
                        rd.rdsplit_set_time(sim.h, 0.0, 0)
                        rd.rdsplit_engine_add(eng, sim.h, w.t_end, w.seed)
                        rd.rdsplit_engine_step(eng, n)

                    ms.append(_timed(batched, stream))
                finally:
                    rd.rdsplit_engine_destroy(eng)
            results.append({"form": "engine", "cluster": cluster, "ms": min(ms[1:]), "periods": n})
    finally:
        sim.close()
    dense_best = pick([r for r in results if r["form"] == "dense"])
    engine_best = pick([r for r in results if r["form"] == "engine"])
    out = {"best": {"mode": dense_best["mode"], "block": dense_best["block"]},
           "single_mesh": "engine" if engine_best and engine_best["ms"] < dense_best["ms"] else "dense",
           "results": results}
    if use_cache:
        cache_put(key, out)
    return out


def tune_engine(rd, sims, t_ends, seeds, reset, stream, clusters=(2, 4, 8, 1), use_cache: bool = True,
                shape_key: str = "") -> dict:
    """CTAs per simulation of the batched engine on the caller's ensemble:
    one full launch per candidate (after `reset()` restores the initial
    state).  Returns {"best": {"cluster": c}, "results": [...]}."""
    key = f"{_device_name()}|engine|{shape_key}"
    if use_cache and shape_key:
        hit = cache_get(key)
        if hit:
            return dict(hit, cached=True)
    results = []
    for c in clusters:
        eng = rd.rdsplit_engine_create(len(sims), sum(rd.rdsplit_get_shape(s.h)[0] for s in sims))
        try:
            rd.rdsplit_engine_set_stream(eng, stream)
            rd.rdsplit_engine_set_concurrency(eng, 0, c)

            def launch():
                for s, te, sd in zip(sims, t_ends, seeds):
                    rd.rdsplit_engine_add(eng, s.h, te, sd)
                rd.rdsplit_engine_step(eng, 1 << 40)
                rd.rdsplit_engine_poll(eng, 1 << 16)

            reset()
            ms = _timed(launch, stream)
            in_flight, _, fit = rd.rdsplit_engine_schedule(eng)
            results.append({"cluster": c, "in_flight": in_flight, "clusters_fit": fit, "ms": ms})
        finally:
            rd.rdsplit_engine_destroy(eng)
    best = pick(results)
    out = {"best": {"cluster": best["cluster"]}, "results": results}
    if use_cache and shape_key:
        cache_put(key, out)
    return out
