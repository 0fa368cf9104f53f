#!/usr/bin/env python3
"""Throughput benchmark of the operator-splitting hot path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

One *step* advances the whole workload from its initial state to t_end
(every period of Algorithm 1: reactions, mean-corrected diffusion count,
multinomial split, synchronous transfer).  The metric is tet-period updates
per second (one tet advanced through one period, all species).

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the stream the library launches on; L2 is flushed (256 MiB write) between
steps, outside the events; barrier + synchronize on both sides; the maximum
over ranks is reported.  Under torchrun each rank runs its own replica of
the workload (weak scaling, no collective on the data path).

Printed: one JSON line (rank 0) with the metric, the roofline of the period
kernel (algorithmic bytes per launch / CUDA-event duration of sampled
launches), the SM clocks sampled during the timed region, an end-to-end
figure through the C ABI with host buffers, and the serial oracle timed on a
bounded sample on the host cores (``cpu_baseline``).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "tet-period updates/s"
UNIT = "tet-period/s"


# --------------------------------------------------------------- workloads --

def engine_bytes_per_entry(S: int) -> int:
    """Algorithmic bytes per processed (simulation, tet) entry of the batched
    engine, counted as for one tet-period of the fused period kernel: the
    reverse-face table (16) and, per species, the kept count (read 4, write
    4), the four incoming and the four outgoing transfers (16 + 16) and the
    cumulative face thresholds (16): 16 + 56 S."""
    return 16 + 56 * S


def make_workload(name: str):
    from paper_1512_03126_gb300 import inputs as I
    if name == "rd48k":
        return I.config_reaction_diffusion_48k()
    if name == "diffusion3072":
        return I.config_diffusion_3072()
    if name == "bar":
        return I.config_bar()
    raise SystemExit(f"unknown workload {name}")


def algorithmic_bytes_per_tet_period(S: int, R: int, masked: bool) -> int:
    """Bytes the fused period kernel must move per tet and period: the
    reverse-face table (16 B) and, per species, the remaining count (read 4,
    write 4), the four incoming out-slots (16), the four outgoing out-slots
    (16) and the cumulative face thresholds (16); with reactions the tet
    volume (8) and, with a reaction mask, its bits (4)."""
    return 16 + 56 * S + (8 if R > 0 else 0) + (4 if masked else 0)


def host_cores() -> int:
    """Cores this process may run on: the affinity mask, capped by a cgroup
    (v2) CPU quota when one is set."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        quota, period = open("/sys/fs/cgroup/cpu.max").read().split()[:2]
        if quota != "max":
            n = max(1, min(n, int(int(quota) / int(period))))
    except (OSError, ValueError):
        pass
    return n


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- ours ---

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1512_03126_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()
    from paper_1512_03126_gb300 import rdsplit as rd

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload)
    T, S, R = w.mesh.n_tets, w.model.n_species, w.model.n_reactions
    stream = torch.cuda.current_stream()
    sim = rd.Simulation(w.mesh, w.model, stream=stream)
    rd.rdsplit_set_period_kernel(sim.h, args.period_mode, args.period_block)
    from paper_1512_03126_gb300 import dist as D
    seed = D.rank_seed(w.seed, rank)
    d_init = torch.from_numpy(np.ascontiguousarray(w.counts)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step():
        rd.rdsplit_set_counts_device(sim.h, d_init)
        rd.rdsplit_set_time(sim.h, 0.0, 0)
        sim.run(w.t_end, seed)

    for _ in range(args.warmup):
        step()
    _, periods = sim.time
    tau = sim.tau
    units_per_step = T * periods

    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = rd.rdsplit_kernel_launches()
    rd.rdsplit_set_timing(sim.h, 16)
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = rd.rdsplit_kernel_launches() - launches0
    kms, kn = rd.rdsplit_get_timing(sim.h)
    rd.rdsplit_set_timing(sim.h, 0)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = D.max_over_ranks(total_ms, dev)
    seconds = total_ms / 1e3
    value = units_per_step * args.steps * world / seconds

    # roofline of the period kernel
    bpt = algorithmic_bytes_per_tet_period(S, R, w.model.mask is not None)
    per_launch_s = (kms / kn) / 1e3 if kn else float("nan")
    achieved = bpt * T / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    two, blk = rd.rdsplit_get_period_kernel(sim.h)
    kname = f"k_period_light (block {blk}) + k_period_slow" if two else f"k_period (block {blk})"
    roofline = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "bytes_per_tet_period": bpt, "launch_us": round(per_launch_s * 1e6, 3),
                "sampled_launches": kn, "peak_source": f"{peak_kind} hbm_gbs"}

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(np.ascontiguousarray(w.counts)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        hin, hout = host_in.numpy(), host_out.numpy()
        for _ in range(1):
            rd.rdsplit_set_counts(sim.h, hin)
            rd.rdsplit_set_time(sim.h, 0.0, 0)
            sim.run(w.t_end, seed)
            rd.rdsplit_get_counts(sim.h, hout)
        e_ms = 0.0
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rd.rdsplit_set_counts(sim.h, hin)
            rd.rdsplit_set_time(sim.h, 0.0, 0)
            sim.run(w.t_end, seed)
            rd.rdsplit_get_counts(sim.h, hout)
            e1.record(stream)
            e1.synchronize()
            e_ms += e0.elapsed_time(e1)
        e2e = {"value": units_per_step * n_e2e * world / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(hin.nbytes), "d2h_bytes_per_step": int(hout.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    sim.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32 counts, f64 rates",
        "data": "synthetic (seeded Kuhn-cube mesh and placement)",
        "config": {"workload": w.name, "n_tets": T, "species": S, "reactions": R, "t_end_s": w.t_end,
                   "periods": periods, "tau_s": tau, "tet_periods_per_step": units_per_step,
                   "l2": "flushed between steps (256 MiB write); the 10 MB state stays L2-resident "
                         "across the periods of a step by design",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "cpu_baseline": cpu,
    }


def cpu_baseline(w, seconds: float):
    """The serial oracle, as it stands, on the host: a bounded number of
    periods of the same workload, scaled to tet-period updates/s."""
    from oracle import oracle as O
    O.lib()
    t0 = time.perf_counter()
    O.run(w.mesh, w.model, w.counts, w.t_end, w.seed, max_periods=5)
    per_period = (time.perf_counter() - t0) / 5
    n = max(5, int(seconds / max(per_period, 1e-6)))
    t0 = time.perf_counter()
    _, _, p = O.run(w.mesh, w.model, w.counts, w.t_end, w.seed, max_periods=n)
    dt = time.perf_counter() - t0
    return {"value": w.mesh.n_tets * p / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {p} periods of {w.name} ({w.mesh.n_tets} tets), one host core, {dt:.1f} s"}


# ---------------------------------------------------------------- ensemble --

def run_ensemble(args, rank, world, local_rank):
    """512 independent simulations (n^3*6 jittered cubes, n ~ U{6..40}), each
    run from its initial state to t_end = 0.1 s: batched in the persistent
    engine (one launch for all of them) against the plain form (each
    simulation's own launch sequence through rdsplit_run)."""
    import torch
    from paper_1512_03126_gb300 import build, inputs as I
    build.build()
    from paper_1512_03126_gb300 import rdsplit as rd
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sizes = I.ensemble_sizes()
    n_inst = len(sizes) if args.instances <= 0 else min(args.instances, len(sizes))
    t0 = time.perf_counter()
    ws = [I.ensemble_instance(i, int(sizes[i]), args.ensemble_t_end) for i in range(n_inst)]
    gen_s = time.perf_counter() - t0
    from paper_1512_03126_gb300 import dist as D
    seeds = [D.rank_seed(w.seed, rank) for w in ws]
    sims = [rd.Simulation(w.mesh, w.model, stream=stream) for w in ws]
    inits = [torch.from_numpy(np.ascontiguousarray(w.counts)).to(dev) for w in ws]
    total_tets = sum(w.mesh.n_tets for w in ws)
    periods = []
    for w, s in zip(ws, sims):
        tau = s.tau
        t, P = 0.0, 0
        while t < w.t_end:
            t = w.t_end if t + tau > w.t_end else t + tau
            P += 1
        periods.append(P)
    units = sum(w.mesh.n_tets * P for w, P in zip(ws, periods))
    eng = rd.rdsplit_engine_create(n_inst, total_tets)
    rd.rdsplit_engine_set_stream(eng, stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def reset():
        for s, x in zip(sims, inits):
            rd.rdsplit_set_counts_device(s.h, x)
            rd.rdsplit_set_time(s.h, 0.0, 0)

    def batched():
        for s, w, sd in zip(sims, ws, seeds):
            rd.rdsplit_engine_add(eng, s.h, w.t_end, sd)
        rd.rdsplit_engine_step(eng, 1 << 40)
        rd.rdsplit_engine_poll(eng, 1 << 16)

    # CTAs per simulation, chosen by timing one launch of each shape (untimed)
    tuned = None
    if not args.no_autotune:
        from paper_1512_03126_gb300 import autotune
        tuned = autotune.tune_engine(rd, sims, [w.t_end for w in ws], seeds, reset, stream, use_cache=False)
        by = {r["cluster"]: r["ms"] for r in tuned["results"]}
        tuned.update({"default_cluster": 2, "default_ms": by.get(2), "chosen_cluster": tuned["best"]["cluster"],
                      "chosen_ms": by.get(tuned["best"]["cluster"])})
        rd.rdsplit_engine_set_concurrency(eng, 0, tuned["best"]["cluster"])

    for _ in range(args.warmup):
        reset()
        batched()
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = rd.rdsplit_kernel_launches()
    steps0, proc0, _, _ = rd.rdsplit_engine_stats(eng)
    rd.rdsplit_engine_set_timing(eng, 1)
    total_ms = 0.0
    for _ in range(args.steps):
        reset()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batched()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = rd.rdsplit_kernel_launches() - launches0
    steps1, proc1, kms, kn = rd.rdsplit_engine_stats(eng)
    slot_times = rd.rdsplit_engine_slot_times(eng, n_inst)   # the last timed launch
    rd.rdsplit_engine_set_timing(eng, 0)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms = D.max_over_ranks(total_ms, dev)
    value = units * args.steps * world / (total_ms / 1e3)
    gsteps = (steps1 - steps0) / args.steps
    entries = (proc1 - proc0) / args.steps
    bpe = engine_bytes_per_entry(1)
    per_launch_s = (kms / kn) / 1e3 if kn else float("nan")
    launches_per_step = kn / args.steps if args.steps else 1
    achieved = bpe * (entries / launches_per_step) / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    roofline = {"kernel": "k_engine_run", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "bytes_per_entry": bpe, "entries_per_launch": round(entries / launches_per_step, 1),
                "launch_us": round(per_launch_s * 1e6, 3), "sampled_launches": kn,
                "peak_source": f"{peak_kind} hbm_gbs",
                "limit": "not HBM: DRAM moves ~2 B per entry (L2 serves the active tets); instruction issue "
                         "and the per-period cluster barrier bound it"}

    in_flight, csize, fit = rd.rdsplit_engine_schedule(eng)
    tail = engine_tail(slot_times, periods, [w.mesh.n_tets for w in ws], in_flight)
    tail.update({"cluster_ctas": csize, "clusters_fit": fit})

    # the plain form: each simulation through its own rdsplit_run
    plain = None
    if rank == 0 and not args.no_plain:
        reset()
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s, w, sd in zip(sims, ws, seeds):
            s.run(w.t_end, sd)
        e1.record(stream)
        e1.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": units / (pms / 1e3), "unit": UNIT, "ms": pms,
                 "launches": sum(periods) + 2 * n_inst,
                 "form": "one rdsplit_run launch sequence per simulation (dense period kernel)"}

    # the plain engine form: the same engine, one simulation per launch
    # (4-CTA clusters, the fastest of 1, 2 and 4 CTAs for one simulation), on every 8th
    # instance; separates the gain of batching from that of skipping empty tets
    plain_engine = None
    if rank == 0 and not args.no_plain:
        sample = list(range(0, n_inst, args.plain_engine_stride))
        e1 = rd.rdsplit_engine_create(1, max(w.mesh.n_tets for w in ws))
        rd.rdsplit_engine_set_stream(e1, stream)
        rd.rdsplit_engine_set_concurrency(e1, 1, 4)
        reset()
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e9 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in sample:
            rd.rdsplit_engine_add(e1, sims[i].h, ws[i].t_end, seeds[i])
            rd.rdsplit_engine_step(e1, 1 << 40)
            rd.rdsplit_engine_poll(e1, 4)
        e9.record(stream)
        e9.synchronize()
        pe_ms = e0.elapsed_time(e9)
        rd.rdsplit_engine_destroy(e1)
        pe_units = sum(ws[i].mesh.n_tets * periods[i] for i in sample)
        plain_engine = {"value": pe_units / (pe_ms / 1e3), "unit": UNIT, "ms": pe_ms, "instances": len(sample),
                        "form": f"one engine launch per simulation (4-CTA cluster), every "
                                f"{args.plain_engine_stride}th instance"}

    # end to end: host counts in, host counts out, through the public calls
    e2e = None
    if not args.no_e2e:
        host_in = [torch.from_numpy(np.ascontiguousarray(w.counts)).pin_memory() for w in ws]
        host_out = [torch.empty_like(x).pin_memory() for x in host_in]
        e_ms = []
        for _ in range(max(3, min(args.steps, 5))):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for s, x in zip(sims, host_in):
                rd.rdsplit_set_counts(s.h, x.numpy())
                rd.rdsplit_set_time(s.h, 0.0, 0)
            rd.rdsplit_ensemble_run([s.h for s in sims], [w.t_end for w in ws], seeds)
            for s, y in zip(sims, host_out):
                rd.rdsplit_get_counts(s.h, y.numpy())
            e1.record(stream)
            e1.synchronize()
            e_ms.append(e0.elapsed_time(e1))
        nb = sum(int(x.numel()) * 4 for x in host_in)
        e_ms = D.max_over_ranks(sum(e_ms), dev) / len(e_ms) if world > 1 else sum(e_ms) / len(e_ms)
        e2e = {"value": units * world / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb, "steps": max(3, min(args.steps, 5)), "ms_per_step": e_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.lib()
        t0 = time.perf_counter()
        done, k = 0, 0
        while time.perf_counter() - t0 < args.cpu_seconds and k < n_inst:
            w = ws[k]
            _, _, p = O.run(w.mesh, w.model, w.counts, w.t_end, seeds[k], max_periods=args.cpu_periods)
            done += w.mesh.n_tets * p
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
               "host_cores": host_cores(),
               "sample": f"first {args.cpu_periods} periods of instances 0..{k - 1} of the ensemble, "
                         f"one host core, {dt:.1f} s"}

    rd.rdsplit_engine_destroy(eng)
    for s in sims:
        s.close()
    configs = None
    if rank == 0 and not args.no_configs:
        configs = run_configs(args, stream, flush)
    reorder = None
    if rank == 0 and not args.no_reorder:
        reorder = run_reorder(args, stream, flush)
    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(args, stream)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32 counts, f64 rates",
        "data": "synthetic (seeded jittered Kuhn cubes, point-source initial state)",
        "config": {"workload": f"batched ensemble of {n_inst} cubes n^3*6, n~U{{6..40}}, t_end {args.ensemble_t_end} s",
                   "instances": n_inst, "tets": total_tets, "tet_periods_per_step": units,
                   "engine_periods_per_step": gsteps, "periods_sum": sum(periods), "periods_max": max(periods),
                   "processed_entries_per_step": entries, "mesh_generation_s": round(gen_s, 1),
                   "l2": "flushed between steps (256 MiB write); per step the ensemble state is 2.3 GB",
                   "parallelism": f"replicas x{world} (each rank its own ensemble, own seeds)"},
        "processed_entries_per_s": entries * args.steps * world / (total_ms / 1e3),
        "roofline": roofline, "tail": tail, "autotune": tuned, "plain": plain,
        "batched_vs_plain": (value / plain["value"]) if plain else None,
        "plain_engine": plain_engine,
        "batched_vs_plain_engine": (value / plain_engine["value"]) if plain_engine else None,
        "serving": serving, "configs": configs, "reorder": reorder,
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "cpu_baseline": cpu,
    }


def engine_tail(slot_times, periods, tets, in_flight: int) -> dict:
    """How the engine's time splits, from each simulation's device-clock
    start and end and its processed entries (one launch): the share of the
    launch with fewer simulations running than clusters in flight, the mean
    number running, the longest simulation, and a least-squares split of the
    simulations' spans into a cost per period and a cost per entry."""
    st = np.asarray(slot_times, dtype=np.float64)
    ok = (st[:, 0] > 0) & (st[:, 1] >= st[:, 0])
    if not ok.any():
        return None
    idx = np.nonzero(ok)[0]
    st = st[ok]
    P = np.asarray(periods, dtype=np.float64)[idx]
    t0, t1 = st[:, 0].min(), st[:, 1].max()
    ev = sorted([(a, 1) for a in st[:, 0]] + [(b, -1) for b in st[:, 1]])
    busy, last, under, area, peak = 0, t0, 0.0, 0.0, 0
    for t, d in ev:
        if busy < in_flight:
            under += t - last
        area += busy * (t - last)
        busy += d
        peak = max(peak, busy)
        last = t
    span = st[:, 1] - st[:, 0]
    i = int(np.argmax(span))
    A = np.stack([P, st[:, 2]], axis=1)
    coef, *_ = np.linalg.lstsq(A, span, rcond=None)
    dur = t1 - t0 if t1 > t0 else 1.0
    return {"launch_ms": dur / 1e6, "in_flight": in_flight, "max_running": int(peak),
            "mean_running": area / dur, "frac_below_full": under / dur,
            "sum_spans_ms": float(span.sum() / 1e6),
            "us_per_period": float(coef[0] / 1e3), "ns_per_entry": float(coef[1]),
            "longest_sim_ms": float(span[i] / 1e6), "longest_sim_periods": int(P[i]),
            "longest_sim_tets": int(np.asarray(tets)[idx[i]]),
            "last_start_ms": float((st[:, 0].max() - t0) / 1e6)}


def run_reorder(args, stream, flush):
    """The batched engine on meshes numbered at random (as a generator
    without locality would number them): a sub-ensemble of the workload,
    stored in the caller's numbering, stored along the library's Morton
    curve (RDSPLIT_REORDER_SFC), and, for reference, in the generator's own
    Morton numbering.  Device time of one engine launch each."""
    import torch
    from paper_1512_03126_gb300 import inputs as I
    from paper_1512_03126_gb300 import rdsplit as rd
    sizes = I.ensemble_sizes()
    idx = list(range(0, len(sizes), max(1, len(sizes) // args.reorder_instances)))[: args.reorder_instances]
    base = [I.ensemble_instance(i, int(sizes[i]), args.reorder_t_end) for i in idx]
    shuffled = []
    for i, w in zip(idx, base):
        m, _ = I.shuffle_mesh(w.mesh, 100 + i)
        shuffled.append(I.Workload(w.name, m, w.model, I.point_source(m, 1, 0, 6000), w.t_end, w.seed))
    out = {"instances": len(idx), "t_end_s": args.reorder_t_end}
    for label, ws, reorder in (("generator_order_ms", base, False), ("shuffled_ms", shuffled, False),
                               ("shuffled_reordered_ms", shuffled, True)):
        sims = [rd.Simulation(w.mesh, w.model, w.counts, stream=stream, reorder=reorder) for w in ws]
        eng = rd.rdsplit_engine_create(len(ws), sum(w.mesh.n_tets for w in ws))
        rd.rdsplit_engine_set_stream(eng, stream)
        ms = []
        for rep in range(3):
            for s, w in zip(sims, ws):
                rd.rdsplit_set_counts(s.h, w.counts)
                rd.rdsplit_set_time(s.h, 0.0, 0)
                rd.rdsplit_engine_add(eng, s.h, w.t_end, w.seed)
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rd.rdsplit_engine_step(eng, 1 << 40)
            e1.record(stream)
            e1.synchronize()
            rd.rdsplit_engine_poll(eng, 1 << 16)
            if rep:
                ms.append(e0.elapsed_time(e1))
        out[label] = sum(ms) / len(ms)
        rd.rdsplit_engine_destroy(eng)
        for x in sims:
            x.close()
    return out


# ----------------------------------------------------------------- configs --

def time_dense(rd, w, steps: int, warmup: int, stream, flush, mode: int = 0, block: int = 0):
    """One workload through rdsplit_run, from its initial state to t_end per
    step: device time per step (CUDA events, L2 flushed between steps) and
    the roofline of the period kernel from sampled launches."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    sim = rd.Simulation(w.mesh, w.model, stream=stream)
    rd.rdsplit_set_period_kernel(sim.h, mode, block)
    d_init = torch.from_numpy(np.ascontiguousarray(w.counts)).to(dev)

    def step():
        rd.rdsplit_set_counts_device(sim.h, d_init)
        rd.rdsplit_set_time(sim.h, 0.0, 0)
        sim.run(w.t_end, w.seed)

    for _ in range(warmup):
        step()
    _, periods = sim.time
    T, S, R = w.mesh.n_tets, w.model.n_species, w.model.n_reactions
    torch.cuda.synchronize()
    l0 = rd.rdsplit_kernel_launches()
    rd.rdsplit_set_timing(sim.h, 8)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    kms, kn = rd.rdsplit_get_timing(sim.h)
    rd.rdsplit_set_timing(sim.h, 0)
    launches = rd.rdsplit_kernel_launches() - l0
    two, blk = rd.rdsplit_get_period_kernel(sim.h)
    sim.close()
    bpt = algorithmic_bytes_per_tet_period(S, R, w.model.mask is not None)
    per_launch_s = (kms / kn) / 1e3 if kn else float("nan")
    achieved = bpt * T / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    return {"value": T * periods * steps / (total / 1e3), "unit": UNIT, "ms_per_step": total / steps,
            "steps": steps, "periods": periods, "n_tets": T, "species": S, "reactions": R,
            "gpu_launches": launches,
            "roofline": {"kernel": f"k_period_light (block {blk}) + k_period_slow" if two else f"k_period (block {blk})",
                         "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "bytes_per_tet_period": bpt,
                         "launch_us": round(per_launch_s * 1e6, 3), "sampled_launches": kn,
                         "peak_source": f"{peak_kind} hbm_gbs"}}


def oracle_one_core(w, seconds: float):
    """The serial oracle, as it stands, on one host core: the first periods
    of the workload (bounded to about `seconds`), as tet-period updates/s."""
    from oracle import oracle as O
    O.lib()
    t0 = time.perf_counter()
    O.run(w.mesh, w.model, w.counts, w.t_end, w.seed, max_periods=2)
    per = (time.perf_counter() - t0) / 2
    n = max(2, int(seconds / max(per, 1e-6)))
    t0 = time.perf_counter()
    _, _, p = O.run(w.mesh, w.model, w.counts, w.t_end, w.seed, max_periods=n)
    dt = time.perf_counter() - t0
    return {"value": w.mesh.n_tets * p / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {p} periods of {w.name}, one host core, {dt:.1f} s"}


def run_configs(args, stream, flush):
    """The single-mesh workloads through the dense period loop: the
    3,072-tet diffusion cube, the 48,000-tet reaction-diffusion cube and the
    2.4 M-tet bar, each with its roofline and a one-core oracle baseline."""
    from paper_1512_03126_gb300 import inputs as I
    from paper_1512_03126_gb300 import rdsplit as rd
    out = {}
    for name, make, steps in (("diffusion_cube_3072", I.config_diffusion_3072, 5),
                              ("reaction_diffusion_cube_48000", I.config_reaction_diffusion_48k, 3),
                              ("bar_20x20x1000", I.config_bar, 3)):
        t0 = time.perf_counter()
        w = make()
        gen = time.perf_counter() - t0
        default = time_dense(rd, w, steps, 2, stream, flush)
        if args.no_autotune:
            r = default
        else:
            from paper_1512_03126_gb300 import autotune
            tuned = autotune.tune_period(rd, w, stream, use_cache=False)
            best = tuned["best"]
            r = time_dense(rd, w, steps, 2, stream, flush, best["mode"], best["block"])
            r["autotune"] = {"chosen": best, "single_mesh": tuned["single_mesh"], "candidates": tuned["results"],
                             "default": {"kernel": default["roofline"]["kernel"], "value": default["value"],
                                         "ms_per_step": default["ms_per_step"]}}
        r["mesh_generation_s"] = round(gen, 1)
        if not args.no_cpu_baseline:
            r["cpu_baseline"] = oracle_one_core(w, args.config_cpu_seconds)
        out[name] = r
    return out


# ----------------------------------------------------------------- serving --

def run_serving(args, stream):
    """Continuous batching (Poisson arrivals at 200/s, requests drawn from the
    serving generator, 150 GB device budget): p50/p99 latency and throughput,
    the offered load against the throughput reached, and the same requests
    run one after another through rdsplit_run (serial plain)."""
    import torch
    from paper_1512_03126_gb300 import inputs as I, serving as SV
    from paper_1512_03126_gb300 import rdsplit as rd
    reqs = I.serving_requests(args.requests)
    t0 = time.perf_counter()
    prepared = {r.rid: r.workload() for r in reqs}
    gen_s = time.perf_counter() - t0
    # warm the path on two small requests
    small = sorted(reqs, key=lambda r: r.n_tets)[:2]
    warm = SV.Server(150e9, 8, args.slice, stream=stream)
    warm.serve([type(r)(r.rid, 0.0, r.n, r.S, r.t_end, r.model_seed) for r in small], prepared)
    warm.close()
    # CTAs per simulation: the autotuner times the engine on the first
    # requests of the mix (all admitted at once, one launch per cluster size)
    tuned = None
    cluster = args.serve_cluster
    if cluster <= 0:
        from paper_1512_03126_gb300 import autotune
        dev = torch.device("cuda", torch.cuda.current_device())
        head = reqs[:args.serve_tune_requests]
        tsims = [rd.Simulation(prepared[r.rid].mesh, prepared[r.rid].model, stream=stream) for r in head]
        tinit = [torch.from_numpy(np.ascontiguousarray(prepared[r.rid].counts)).to(dev) for r in head]

        def treset():
            for sm, x in zip(tsims, tinit):
                rd.rdsplit_set_counts_device(sm.h, x)
                rd.rdsplit_set_time(sm.h, 0.0, 0)

        try:
            tuned = autotune.tune_engine(rd, tsims, [prepared[r.rid].t_end for r in head],
                                         [prepared[r.rid].seed for r in head], treset, stream,
                                         clusters=(2, 4, 8), use_cache=False)
        finally:
            for sm in tsims:
                sm.close()
        cluster = tuned["best"]["cluster"]
    dense_stream = torch.cuda.Stream() if args.dense_threshold < float("inf") else None
    server = SV.Server(150e9, args.max_slots, args.slice, stream=stream, dense_threshold=args.dense_threshold,
                       dense_stream=dense_stream, dense_lanes=args.dense_lanes, slice_work=args.slice_work,
                       cluster=cluster)
    torch.cuda.synchronize()
    recs = server.serve(reqs, prepared)
    server.close()
    torch.cuda.synchronize()
    out = SV.summarize(recs)
    arrival_span = max(r.arrival for r in reqs) - min(r.arrival for r in reqs)
    offered = out["tet_periods"] / arrival_span if arrival_span > 0 else None
    # serial plain runs of the same requests
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        w = prepared[r.rid]
        with rd.Simulation(w.mesh, w.model, w.counts, stream=stream) as sim:
            sim.run(w.t_end, w.seed)
            sim.counts()
    serial_s = time.perf_counter() - t0
    out.update({"unit": UNIT, "arrival_rate_per_s": 200.0, "arrival_span_s": arrival_span,
                "offered_load": offered,
                "load_vs_throughput": (offered / out["throughput"]) if offered and out["throughput"] else None,
                "saturated": bool(offered and out["throughput"] and offered > 1.2 * out["throughput"]),
                "budget_gb": 150, "slice_periods": args.slice, "slice_work_tet_periods": args.slice_work,
                "dense_lane_threshold_tet_species": args.dense_threshold, "dense_lanes": args.dense_lanes,
                "max_slots": args.max_slots, "cluster_ctas": cluster,
                "cluster_tuning": ({"requests": args.serve_tune_requests, "results": tuned["results"]}
                                   if tuned else None),
                "serial_plain_s": serial_s,
                "serial_plain_throughput": out["tet_periods"] / serial_s,
                "throughput_vs_serial_plain": (out["throughput"] * serial_s / out["tet_periods"]),
                "request_generation_s": round(gen_s, 1), "host_loop_s": server.host_s,
                "latency": "completion - arrival, wall clock, including queueing, upload and read-back"})
    return out


# -------------------------------------------------------------- reference ---

def _oracle_worker(conn, workload: str, index: int, periods: int):
    """One host process of the reference arm: owns one simulation of the
    workload (built before the timed region) and runs `periods` periods of
    the serial oracle on each request."""
    from oracle import oracle as O
    O.lib()
    if workload == "ensemble":
        from paper_1512_03126_gb300 import inputs as I
        sizes = I.ensemble_sizes()
        w = I.ensemble_instance(index, int(sizes[index % len(sizes)]))
    else:
        w = make_workload(workload)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        _, _, p = O.run(w.mesh, w.model, w.counts, w.t_end, w.seed + msg, max_periods=periods)
        conn.send(w.mesh.n_tets * p)


def _reference_all_cores(args, cores: int):
    """Each step: `cores` oracle processes (spawned, one simulation each) run
    args.ref_periods periods at once; returns (tet-periods per step list,
    seconds per step list)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    procs, conns = [], []
    try:
        for c in range(cores):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, args.workload, c, max(1, int(args.ref_periods))),
                            daemon=True)
            p.start()
            procs.append(p)
            conns.append(a)
        for a in conns:
            if a.recv() != "ready":
                raise RuntimeError("oracle worker failed to start")
        done, secs = [], []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            for a in conns:
                a.send(k)
            n = sum(a.recv() for a in conns)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                done.append(n)
                secs.append(dt)
        return done, secs
    finally:
        for a in conns:
            try:
                a.send(None)
            except Exception:
                pass
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()


def run_reference(args, rank, world):
    """The serial oracle timed on the host cores on a bounded sample of the
    same workload per step (the paper's reference implementation is not
    available; this is the CPU restatement of the method).  Every host core
    runs its own simulation (instance c on core c), the ensemble being
    independent simulations; a single-core run is the fallback."""
    if rank != 0:
        return None
    periods_per_step = max(1, int(args.ref_periods))
    cores = host_cores()
    name = "batched ensemble (instance c on host core c)" if args.workload == "ensemble" else args.workload
    try:
        done, secs = _reference_all_cores(args, cores)
    except Exception as e:   # fall back to one core in this process
        print(f"reference arm: all-core run failed ({e}); timing one core", file=sys.stderr)
        cores = 1
        from oracle import oracle as O
        O.lib()
        if args.workload == "ensemble":
            from paper_1512_03126_gb300 import inputs as I
            w = I.ensemble_instance(0, int(I.ensemble_sizes()[0]))
        else:
            w = make_workload(args.workload)
        done, secs = [], []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            _, _, p = O.run(w.mesh, w.model, w.counts, w.t_end, w.seed + k, max_periods=periods_per_step)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                done.append(w.mesh.n_tets * p)
                secs.append(dt)
    total_s = sum(secs)
    value = sum(done) / total_s
    sample = (f"first {periods_per_step} periods of {cores} simulations per step ({name}), "
              f"{cores} host cores, one process each")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32 counts, f64 rates",
            "data": "synthetic", "config": {"workload": name, "periods_per_step": periods_per_step,
                                            "host_cores": cores, "per_core_value": value / cores,
                                            "cpu_model": cpu_model()},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ensemble")
    ap.add_argument("--instances", type=int, default=0, help="ensemble: use the first N instances (0 = all 512)")
    ap.add_argument("--ensemble-t-end", type=float, default=0.1, help="ensemble: simulated time per instance (s)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain-engine-stride", type=int, default=8,
                    help="ensemble: time the one-simulation-per-launch engine on every Nth instance")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--requests", type=int, default=400, help="serving: number of requests")
    ap.add_argument("--slice", type=int, default=256, help="serving: periods per engine launch")
    ap.add_argument("--max-slots", type=int, default=128, help="serving: simulations admitted at once")
    ap.add_argument("--slice-work", type=int, default=20_000_000,
                    help="serving: tet-periods per simulation and engine launch (0: every one advances --slice)")
    ap.add_argument("--dense-threshold", type=float, default=float("inf"),
                    help="serving: n_tets*n_species from which a request runs in a dense lane (inf: none)")
    ap.add_argument("--dense-lanes", type=int, default=2, help="serving: dense lanes")
    ap.add_argument("--serve-cluster", type=int, default=0,
                    help="serving: CTAs per simulation (0: chosen by the autotuner on the first requests)")
    ap.add_argument("--serve-tune-requests", type=int, default=100,
                    help="serving: requests the cluster-size autotuner runs")
    ap.add_argument("--period-mode", type=int, default=0, help="dense period kernel: 0 auto, 1 one pass, 2 two passes")
    ap.add_argument("--period-block", type=int, default=0, help="dense period kernel: block size (0: by mesh size)")
    ap.add_argument("--no-configs", action="store_true", help="skip the single-mesh workloads")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-reorder", action="store_true", help="skip the shuffled-numbering engine measurement")
    ap.add_argument("--reorder-instances", type=int, default=64)
    ap.add_argument("--reorder-t-end", type=float, default=0.02)
    ap.add_argument("--config-cpu-seconds", type=float, default=5.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-periods", type=int, default=300)
    ap.add_argument("--cpu-periods", type=int, default=40)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        import torch
        if world > 1:
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = (run_ensemble if args.workload == "ensemble" else run_ours)(args, rank, world, local_rank)
        if world > 1:
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
