"""Multi-process paths on CPU ranks (gloo, 127.0.0.1).

1. The replica plumbing the benchmark uses under torchrun: distinct seeds
   per rank, round-robin shards that partition the items, and the maximum
   of the per-rank times.
2. The paper's parallel scheme (Sec. III.D, domain decomposition): each rank
   advances its own contiguous range of tets for a period (the oracle's
   per-range Steps 2-3), the out-slots are exchanged once per period, and
   each rank applies what its tets receive.  Because every draw is keyed by
   the canonical tet id, the result must equal the single-process run bit
   for bit, for any number of ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    return dist


def _replica_worker(rank, world, port):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    from paper_1512_03126_gb300 import dist as D
    dist = _init(rank, world, port)
    seeds = torch.tensor([D.rank_seed(7, rank)], dtype=torch.int64)
    allseeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allseeds, seeds)
    assert len({int(x.item()) for x in allseeds}) == world
    items = torch.zeros(50, dtype=torch.int64)
    for i in D.shard(50, rank, world):
        items[i] += 1
    dist.all_reduce(items)
    assert torch.all(items == 1)
    m = D.max_over_ranks(10.0 + rank)
    assert m == 10.0 + world - 1
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_plumbing(world):
    mp.start_processes(_replica_worker, args=(world, _free_port()), nprocs=world, start_method="spawn")


def _dd_workload():
    from paper_1512_03126_gb300 import inputs as I
    m = I.cube(4, 1e-6, 0.2, 12)
    n = I.molecules(20e-6, 1e-18)
    return I.Workload("abc_n4", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4), 1.2e-3, 7)


def _reverse(adj):
    T = adj.shape[0]
    rev = np.full((T, 4), -1, np.int64)
    for t in range(T):
        for f in range(4):
            u = adj[t, f]
            if u >= 0:
                rev[t, f] = int(np.nonzero(adj[u] == t)[0][0])
    return rev


def _dd_worker(rank, world, port, outpath):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    from oracle import oracle as O
    dist = _init(rank, world, port)
    w = _dd_workload()
    T, S = w.mesh.n_tets, w.model.n_species
    bounds = [T * r // world for r in range(world + 1)]
    lo, hi = bounds[rank], bounds[rank + 1]
    width = max(bounds[r + 1] - bounds[r] for r in range(world))
    rev = _reverse(w.mesh.adj)
    N = np.zeros((T, S), np.int32)
    N[lo:hi] = w.counts[lo:hi]            # a rank holds only its own tets
    tau = O.tau(w.mesh, w.model)
    t_now, period = 0.0, 0
    while t_now < w.t_end:
        tau_k, last = tau, False
        if t_now + tau > w.t_end:
            tau_k, last = w.t_end - t_now, True
        out, rem = O.period_tets(w.mesh, w.model, N, period, tau_k, w.seed, lo, hi)
        # the one exchange of the period: every rank's out-slots
        pad = np.zeros((width, S, 4), np.int32)
        pad[:hi - lo] = out
        parts = [torch.zeros((width, S, 4), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(pad))
        full = np.concatenate([parts[r].numpy()[:bounds[r + 1] - bounds[r]] for r in range(world)])
        # synchronous apply for this rank's tets
        N[:] = 0
        for t in range(lo, hi):
            v = rem[t - lo].astype(np.int64)
            for f in range(4):
                u = w.mesh.adj[t, f]
                if u >= 0:
                    v = v + full[u, :, rev[t, f]]
            N[t] = v
        t_now = w.t_end if last else t_now + tau
        period += 1
    mine = torch.from_numpy(np.ascontiguousarray(N[lo:hi]))
    pad = torch.zeros((width, S), dtype=torch.int32)
    pad[:hi - lo] = mine
    parts = [torch.zeros((width, S), dtype=torch.int32) for _ in range(world)]
    dist.all_gather(parts, pad)
    if rank == 0:
        final = np.concatenate([parts[r].numpy()[:bounds[r + 1] - bounds[r]] for r in range(world)])
        np.save(outpath, final)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_domain_decomposition_equals_single_process(oracle, tmp_path, world):
    outpath = str(tmp_path / "dd.npy")
    mp.start_processes(_dd_worker, args=(world, _free_port(), outpath), nprocs=world, start_method="spawn")
    w = _dd_workload()
    ref, _, _ = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
    got = np.load(outpath)
    assert np.array_equal(got, ref)
