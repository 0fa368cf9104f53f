"""Host side of the domain decomposition (Sec. III.D of the paper: each
process advances its own tets for a period, the changes bound for tets of
other processes are buffered, exchanged and applied before the next
period).

A rank owns a contiguous range of tets.  The molecules that its tets send
through a cut face land in the inbox slot 4 u + r of a tet u of another
rank (face r of u); `cut_slots` lists those slots, in increasing order, for
one (sender, receiver) pair of ranges: the sender exports them after each
period and the receiver imports them, in the same order, before the next.
`run_rank` drives one rank of a partitioned run through the library; the
exchange itself is the caller's, and `p2p_exchange` gives one over
torch.distributed point-to-point operations (NCCL between GPUs, with the
buffers left on the device).  No method arithmetic lives here: every period
runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def ranges(n_tets: int, world: int) -> list:
    """Contiguous ranges [lo, hi) of tets per rank, as equal as possible."""
    b = [n_tets * r // world for r in range(world + 1)]
    return [(b[r], b[r + 1]) for r in range(world)]


def cut_slots(adj: np.ndarray, sender: tuple, receiver: tuple) -> np.ndarray:
    """Inbox slots 4 u + r with u in the receiver's range and adj[u][r] in the
    sender's range (int32, increasing)."""
    lo, hi = receiver
    slo, shi = sender
    a = np.asarray(adj[lo:hi])
    u, r = np.nonzero((a >= slo) & (a < shi))
    return ((u + lo) * 4 + r).astype(np.int32)


def run_rank(rd, h, adj, rank: int, parts: list, t_end: float, seed: int, exchange) -> int:
    """Advance this rank's tets of handle h (counts already set) to t_end.
    After every period, for every other rank p with cut faces, the library
    exports the slots this rank's tets filled in p's tets and `exchange`
    sends them, receives what p's tets sent to this rank's tets, and the
    library imports it.  exchange(sends, recvs) takes {p: device int32
    tensor [n][S]} to send and {p: (n, S)} to receive, and returns {p: device
    int32 tensor [n][S]}.  Returns the number of periods."""
    import torch
    _, S = rd.rdsplit_get_shape(h)
    me = parts[rank]
    rd.rdsplit_partition_set(h, me[0], me[1])
    out_slots, in_slots = {}, {}
    for p, rng in enumerate(parts):
        if p == rank:
            continue
        so = cut_slots(adj, me, rng)
        si = cut_slots(adj, rng, me)
        if len(so):
            out_slots[p] = torch.from_numpy(so).cuda()
        if len(si):
            in_slots[p] = torch.from_numpy(si).cuda()
    periods = 0
    more = True
    while more:
        more = rd.rdsplit_partition_step(h, t_end, seed)
        periods += 1
        sends = {}
        for p, sl in out_slots.items():
            buf = torch.empty((sl.numel(), S), dtype=torch.int32, device="cuda")
            sends[p] = rd.rdsplit_inbox_export(h, sl, buf)
        recvs = exchange(sends, {p: (sl.numel(), S) for p, sl in in_slots.items()})
        for p, sl in in_slots.items():
            rd.rdsplit_inbox_import(h, sl, recvs[p])
    rd.rdsplit_partition_end(h)
    return periods


def p2p_exchange(dist, device=None):
    """An `exchange` for run_rank over torch.distributed point-to-point
    operations.  All sends and receives of one period are posted in one
    batch (batch_isend_irecv, one NCCL group between GPUs, so that two ranks
    sending to each other do not wait on each other's order) and completed
    before it returns.  A receive lands in a new int32 tensor on `device`
    (default: the current CUDA device, else the CPU).  With NCCL, completion
    orders the current torch stream after the transfers: the library's
    stream must be that stream (the default), or be synchronised with it,
    before rdsplit_inbox_import reads the buffers."""
    import torch

    def exchange(sends, recv_shapes):
        dev = device
        if dev is None:
            dev = (torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available()
                   else torch.device("cpu"))
        ops, recvs = [], {}
        for p in sorted(set(sends) | set(recv_shapes)):
            if p in recv_shapes:
                recvs[p] = torch.empty(tuple(recv_shapes[p]), dtype=torch.int32, device=dev)
                ops.append(dist.P2POp(dist.irecv, recvs[p], p))
            if p in sends:
                ops.append(dist.P2POp(dist.isend, sends[p].contiguous(), p))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return recvs

    return exchange
