"""Write tests/golden/oracle_runs.json: SHA-256 of the serial oracle's final
counts for the full-size workloads (and a few prefixes), so that GPU parity
at full size can be checked without rerunning the oracle for minutes.

Calls only ``oracle/`` and the seeded input generators.  Usage:
    python tests/golden/make_golden.py [name ...]
    python tests/golden/make_golden.py --check [--max-seconds S] [name ...]
The second form writes nothing: it reruns the stored entries (those named,
else every one whose recorded oracle time is at most S seconds, default 3)
with the oracle built on this host and compares their digests with the
stored ones, so that the oracle's bit-identity across hosts (x86-64 and
aarch64) can be checked; it exits 1 on any mismatch.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_runs.json")


def counts_digest(c) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(c, dtype="<i4").tobytes()).hexdigest()


def entries():
    from paper_1512_03126_gb300 import inputs as I
    sizes = I.ensemble_sizes()
    e = {
        "diffusion_cube_3072": ("diffusion", {}, -1),
        "reaction_diffusion_cube_48000": ("rd48k", {}, -1),
        "reaction_diffusion_cube_48000@300": ("rd48k", {}, 300),
        "bar_20x20x1000@20": ("bar", {}, 20),
        "bar_20x20x1000": ("bar", {}, -1),
    }
    seen = set()
    for i, n in enumerate(sizes):
        if int(n) not in seen:
            seen.add(int(n))
            e[f"ensemble_{i}_n{int(n)}"] = ("ensemble", {"i": i, "n": int(n)}, -1)
    reqs = 0
    for r in I.serving_requests(64):
        if r.n <= 16 and reqs < 12:
            e[f"request_{r.rid}_n{r.n}_S{r.S}"] = ("request", {"rid": r.rid}, -1)
            reqs += 1
    # larger serving requests, stratified over the mesh sizes up to n = 60
    # and the species counts 1..8; eleven of them have n_tets * n_species
    # >= 1e6 and run in the server's dense lane
    for r in I.serving_requests(64):
        if r.rid in LARGE_REQUESTS:
            e[f"request_{r.rid}_n{r.n}_S{r.S}"] = ("request", {"rid": r.rid}, -1)
    return e


# request ids of the serving generator's first 64 requests with stored runs
# beyond the twelve smallest: n 17-25 (31, 29, 47, 59, 35), 26-35 (36, 40,
# 41, 63), 36-45 (27, 19, 10, 0, 45, 6) and 46-60 (55, 57, 24, 49)
LARGE_REQUESTS = (31, 29, 47, 59, 35, 36, 40, 41, 63, 27, 19, 10, 0, 45, 6, 55, 57, 24, 49)


def build_workload(kind, args):
    from paper_1512_03126_gb300 import inputs as I
    if kind == "diffusion":
        return I.config_diffusion_3072()
    if kind == "rd48k":
        return I.config_reaction_diffusion_48k()
    if kind == "bar":
        return I.config_bar()
    if kind == "ensemble":
        return I.ensemble_instance(args["i"], args["n"])
    if kind == "request":
        return I.serving_requests(64)[args["rid"]].workload()
    raise ValueError(kind)


def run_entry(item):
    name, (kind, args, max_periods) = item
    from oracle import oracle as O
    w = build_workload(kind, args)
    t0 = time.time()
    c, t, p = O.run(w.mesh, w.model, w.counts, w.t_end, w.seed, max_periods=max_periods)
    return name, {"sha256": counts_digest(c), "totals": [int(x) for x in c.sum(0)], "t": t, "period": p,
                  "n_tets": w.mesh.n_tets, "n_species": w.model.n_species, "max_periods": max_periods,
                  "oracle_seconds": round(time.time() - t0, 2), "kind": kind, "args": args}


def main(names):
    from oracle import build
    build.build()
    todo = entries()
    if names:
        todo = {k: v for k, v in todo.items() if k in names}
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    # longest first (roughly: the full bar, then requests by size)
    def cost(kv):
        kind, args, maxp = kv[1]
        if kind == "bar" and maxp < 0:
            return -1e30
        if kind == "request":
            r = I.serving_requests(64)[args["rid"]]
            return -float(r.n_tets * r.S * r.t_end)
        return 0.0
    from paper_1512_03126_gb300 import inputs as I
    order = sorted(todo.items(), key=cost)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        for name, rec in pool.imap_unordered(run_entry, order):
            data[name] = rec
            with open(OUT + ".tmp", "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(OUT + ".tmp", OUT)
            print(name, rec["oracle_seconds"], "s", flush=True)


def check(names, max_seconds: float) -> int:
    from oracle import build
    build.build()
    stored = json.load(open(OUT))
    todo = entries()
    pick = names or [k for k, v in stored.items() if v["oracle_seconds"] <= max_seconds]
    order = [(k, todo[k]) for k in sorted(pick) if k in todo and k in stored]
    bad = 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        for name, rec in pool.imap_unordered(run_entry, order):
            ok = rec["sha256"] == stored[name]["sha256"]
            bad += 0 if ok else 1
            print(name, "same" if ok else "DIFFERENT", flush=True)
    print(f"{len(order) - bad} of {len(order)} stored runs reproduced on this host", flush=True)
    return 1 if bad else 0


if __name__ == "__main__":
    argv = sys.argv[1:]
    if argv and argv[0] == "--check":
        argv = argv[1:]
        limit = 3.0
        if len(argv) >= 2 and argv[0] == "--max-seconds":
            limit = float(argv[1])
            argv = argv[2:]
        sys.exit(check(argv, limit))
    main(argv)
