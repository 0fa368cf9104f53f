"""Multi-process paths on CPU ranks (gloo, 127.0.0.1).

1. The replica plumbing the benchmark uses under torchrun: distinct seeds
   per rank, round-robin shards that partition the items, and the maximum
   of the per-rank times.
2. The paper's parallel scheme (Sec. III.D, domain decomposition): each rank
   advances its own contiguous range of tets for a period (the oracle's
   per-range Steps 2-3), the transfers across cut faces (and only those) go
   to the rank that owns the receiving tet once per period, in the order of
   partition.cut_slots, through partition.p2p_exchange (the exchange the
   library offers for NCCL between GPUs, here over gloo), and each rank
   applies what its tets receive.  Because every draw is keyed by
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
    from paper_1512_03126_gb300 import partition as P
    dist = _init(rank, world, port)
    w = _dd_workload()
    T, S = w.mesh.n_tets, w.model.n_species
    adj = w.mesh.adj
    parts = P.ranges(T, world)
    lo, hi = parts[rank]
    rev = _reverse(adj)
    # face f of the writer t = adj[u][r] that points at u
    face_to = lambda t, u: int(np.nonzero(adj[t] == u)[0][0])
    sends = {p: P.cut_slots(adj, (lo, hi), parts[p]) for p in range(world) if p != rank}
    recvs = {p: P.cut_slots(adj, parts[p], (lo, hi)) for p in range(world) if p != rank}
    exchange = P.p2p_exchange(dist, torch.device("cpu"))
    N = np.zeros((T, S), np.int32)
    N[lo:hi] = w.counts[lo:hi]            # a rank holds only its own tets
    tau = O.tau(w.mesh, w.model)
    t_now, period = 0.0, 0
    while t_now < w.t_end:
        tau_k, last = tau, False
        if t_now + tau > w.t_end:
            tau_k, last = w.t_end - t_now, True
        out, rem = O.period_tets(w.mesh, w.model, N, period, tau_k, w.seed, lo, hi)
        # the one exchange of the period: the transfers across cut faces
        # only, to the rank that owns the receiving tet (the library's
        # point-to-point exchange, here over gloo with host tensors)
        bufs = {}
        for p, sl in sends.items():
            if not len(sl):
                continue
            buf = np.zeros((len(sl), S), np.int32)
            for k, slot in enumerate(sl):
                u, r = divmod(int(slot), 4)
                t = int(adj[u, r])
                buf[k] = out[t - lo, :, face_to(t, u)]
            bufs[p] = torch.from_numpy(buf)
        got = exchange(bufs, {p: (len(sl), S) for p, sl in recvs.items() if len(sl)})
        incoming = np.zeros((T, S), np.int64)
        for p, x in got.items():
            for k, slot in enumerate(recvs[p]):
                u = int(slot) // 4
                incoming[u] += x.numpy()[k]
        # synchronous apply for this rank's tets
        N[:] = 0
        for t in range(lo, hi):
            v = rem[t - lo].astype(np.int64) + incoming[t]
            for f in range(4):
                u = adj[t, f]
                if lo <= u < hi:
                    v = v + out[u - lo, :, rev[t, f]]
            N[t] = v
        t_now = w.t_end if last else t_now + tau
        period += 1
    width = max(b - a for a, b in parts)
    pad = torch.zeros((width, S), dtype=torch.int32)
    pad[:hi - lo] = torch.from_numpy(np.ascontiguousarray(N[lo:hi]))
    allparts = [torch.zeros((width, S), dtype=torch.int32) for _ in range(world)]
    dist.all_gather(allparts, pad)
    if rank == 0:
        final = np.concatenate([allparts[r].numpy()[:parts[r][1] - parts[r][0]] for r in range(world)])
        np.save(outpath, final)
    dist.destroy_process_group()


def test_cut_slots_pair_up():
    """Each cut face appears once, in the sender's export list and in the
    receiver's import list (the same list), and only cut faces do."""
    from paper_1512_03126_gb300 import partition as P
    w = _dd_workload()
    adj = w.mesh.adj
    parts = P.ranges(w.mesh.n_tets, 3)
    seen = set()
    for a in range(3):
        for b in range(3):
            if a == b:
                continue
            sl = P.cut_slots(adj, parts[a], parts[b])
            assert np.all(np.diff(sl) > 0)
            for slot in sl:
                u, r = divmod(int(slot), 4)
                assert parts[b][0] <= u < parts[b][1] and parts[a][0] <= adj[u, r] < parts[a][1]
                seen.add(int(slot))
    cut = {4 * u + r for u in range(w.mesh.n_tets) for r in range(4)
           if adj[u, r] >= 0 and [lo <= u < hi for lo, hi in parts] != [lo <= adj[u, r] < hi for lo, hi in parts]}
    assert seen == cut


@pytest.mark.parametrize("world", [2, 3])
def test_domain_decomposition_equals_single_process(oracle, tmp_path, world):
    outpath = str(tmp_path / "dd.npy")
    mp.start_processes(_dd_worker, args=(world, _free_port(), outpath), nprocs=world, start_method="spawn")
    w = _dd_workload()
    ref, _, _ = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
    got = np.load(outpath)
    assert np.array_equal(got, ref)
