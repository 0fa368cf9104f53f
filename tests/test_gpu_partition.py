"""Domain decomposition through the library (Sec. III.D): two or three
processes on one GPU, each advancing its own range of tets with
rdsplit_partition_step and exchanging only the transfers across cut faces
(rdsplit_inbox_export / rdsplit_inbox_import) through gloo on the host once
per period.  Every draw is keyed by canonical tet ids, so the ranks'
counts together equal one process's rdsplit_run, and the oracle's, bit for
bit.  No kernel waits on another process: the host drives the exchange
between launches."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1512_03126_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(kind):
    if kind == "abc":
        m = I.cube(6, 1e-6, 0.2, 12)
        n = I.molecules(20e-6, 1e-18)
        return I.Workload("abc_n6", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4), 1.2e-3, 7)
    bar = I.kuhn_box(4, 4, 40, (0.2e-6, 0.2e-6, 2e-6), 0.2, 13)
    bm = I.bar_model(bar)
    V = 0.2e-6 * 0.2e-6 * 2e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    return I.Workload("bar_small", bar, bm, I.place_by_volume(bar, [f, f, f, b, b, 0, 0, 0], 5), 1.0e-3, 9)


def _rank(rank, world, port, kind, outpath):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_1512_03126_gb300 import partition as P
    from paper_1512_03126_gb300 import rdsplit as rd
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = _workload(kind)
    T, S = w.mesh.n_tets, w.model.n_species
    parts = P.ranges(T, world)

    def exchange(sends, recv_shapes):
        reqs, host = [], {}
        for p, buf in sends.items():
            reqs.append(dist.isend(buf.cpu(), dst=p))
        for p, shape in recv_shapes.items():
            host[p] = torch.zeros(shape, dtype=torch.int32)
            reqs.append(dist.irecv(host[p], src=p))
        for q in reqs:
            q.wait()
        return {p: x.cuda() for p, x in host.items()}

    with rd.Simulation(w.mesh, w.model, w.counts) as sim:
        periods = P.run_rank(rd, sim.h, w.mesh.adj, rank, parts, w.t_end, w.seed, exchange)
        mine = sim.counts()[parts[rank][0]:parts[rank][1]]
        t, period = sim.time
    width = max(b - a for a, b in parts)
    pad = torch.zeros((width, S), dtype=torch.int32)
    pad[:len(mine)] = torch.from_numpy(np.ascontiguousarray(mine))
    allparts = [torch.zeros((width, S), dtype=torch.int32) for _ in range(world)]
    dist.all_gather(allparts, pad)
    if rank == 0:
        final = np.concatenate([allparts[r].numpy()[:parts[r][1] - parts[r][0]] for r in range(world)])
        np.save(outpath, final)
        np.save(outpath + ".meta.npy", np.array([periods, period, t]))
    dist.destroy_process_group()


@pytest.mark.parametrize("kind, world", [("abc", 2), ("bar", 3)])
def test_partitioned_run_equals_one_process(oracle, tmp_path, kind, world):
    import torch
    assert torch.cuda.is_available()
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit as rd
    outpath = str(tmp_path / "part.npy")
    mp.start_processes(_rank, args=(world, _free_port(), kind, outpath), nprocs=world, start_method="spawn")
    w = _workload(kind)
    with rd.Simulation(w.mesh, w.model, w.counts) as sim:
        sim.run(w.t_end, w.seed)
        one = sim.counts()
        t1, p1 = sim.time
    ref, _, _ = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
    got = np.load(outpath)
    periods, period, t = np.load(outpath + ".meta.npy")
    assert np.array_equal(one, ref)
    assert np.array_equal(got, ref)
    assert int(periods) == int(period) == p1
