"""The allocation-free entry point, rdsplit_run_static.

It exists for callers that cannot call cudaMalloc (a plugin inside a host
application that owns all device memory, or a real-time loop that must not
stall on an allocation); it keeps every intermediate array in one static
device array.  This test calls it through the C ABI twice in a row, on two
different problems, and checks each result against the handle-based
rdsplit_run on the same inputs.  Counts are integers from keyed random
streams, so the tolerance is zero, as in every other parity test here.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def _problems():
    m = I.cube(5, 1e-6, 0.2, 12)
    n = I.molecules(20e-6, 1e-18)
    abc = I.Workload("abc_n5", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4), 2e-3, 7)
    bar = I.kuhn_box(4, 4, 12, (0.2e-6, 0.2e-6, 0.6e-6), 0.2, 13)
    V = 0.2e-6 * 0.2e-6 * 0.6e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    masked = I.Workload("bar_4x4x12", bar, I.bar_model(bar),
                        I.place_by_volume(bar, [f, f, f, b, b, 0, 0, 0], 5), 1.2e-3, 9)
    return [abc, masked]


def _handle_run(rd, w):
    with rd.Simulation(w.mesh, w.model, w.counts) as sim:
        sim.run(w.t_end, w.seed)
        return sim.counts(), sim.time


def _static_run(rd, w):
    import torch
    dev = torch.device("cuda", 0)
    m, model = w.mesh, w.model
    d_adj = torch.from_numpy(np.ascontiguousarray(m.adj)).to(dev)
    d_vol = torch.from_numpy(np.ascontiguousarray(m.vol)).to(dev)
    d_area = torch.from_numpy(np.ascontiguousarray(m.area)).to(dev)
    d_dist = torch.from_numpy(np.ascontiguousarray(m.dist)).to(dev)
    d_mask = None if model.mask is None else torch.from_numpy(np.ascontiguousarray(model.mask)).to(dev)
    d_counts = torch.from_numpy(np.ascontiguousarray(w.counts)).to(dev)
    torch.cuda.synchronize()
    t, p = rd.rdsplit_run_static(m.n_tets, d_adj, d_vol, d_area, d_dist, model.n_species, model.D,
                                 model.n_reactions, model.lhs, model.rhs, model.k, d_mask, model.tau_scale,
                                 d_counts, 0.0, 0, w.t_end, w.seed)
    return d_counts.cpu().numpy(), (t, p)


def test_static_entry_point_matches_rdsplit_run_twice(rd):
    for w in _problems():
        need = rd.rdsplit_static_scratch_bytes(w.mesh.n_tets, w.model.n_species, w.model.mask is not None)
        assert 0 < need <= rd.RDSPLIT_STATIC_SCRATCH_BYTES
        ref, (tr, pr) = _handle_run(rd, w)
        got, (tg, pg) = _static_run(rd, w)
        assert (tg, pg) == (tr, pr)
        assert np.array_equal(got, ref), f"{w.name}: {np.count_nonzero(got != ref)} counts differ"


def test_static_entry_point_rejects_oversized_problems(rd):
    import torch
    T = 2_000_000
    assert rd.rdsplit_static_scratch_bytes(T, 8, False) > rd.RDSPLIT_STATIC_SCRATCH_BYTES
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(rd.RdsplitError) as e:
        rd.rdsplit_run_static(T, dummy, dummy, dummy, dummy, 8, np.full(8, 1e-12), 0, None, None, None, None,
                              1.0, dummy, 0.0, 0, 1.0, 1)
    assert e.value.code == rd.RDSPLIT_EINVAL
    assert "static maximum" in rd.rdsplit_last_error()
