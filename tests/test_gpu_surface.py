"""Surface (triangle) diffusion on the GPU: a triangulated sheet passed
through the same C ABI (triangle area for the volume, edge length for the
face area, fourth neighbour -1) gives exactly the oracle's counts, dense and
batched (tolerance 0)."""
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


def _workloads():
    m = I.triangle_sheet(40, 40, (4e-6, 4e-6), 0.2, 9)
    diff = I.Workload("sheet_point_source", m, I.diffusion_model(1e-12),
                      I.point_source(m, 1, 0, 6000, where=(2e-6, 2e-6, 0.0)), 0.02, 3)
    decay = I.Model(D=np.array([0.5e-12]), lhs=np.ones((1, 1), np.int32), rhs=np.zeros((1, 1), np.int32),
                    k=np.array([20.0]))
    c = np.full((m.n_tets, 1), 7, np.int32)
    dec = I.Workload("sheet_decay", m, decay, c, 0.03, 4)
    return [diff, dec]


def test_surface_diffusion_bit_exact(rd, oracle):
    ws = _workloads()
    refs = [oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)[0] for w in ws]
    for w, ref in zip(ws, refs):
        with rd.Simulation(w.mesh, w.model, w.counts) as sim:
            assert sim.tau == oracle.tau(w.mesh, w.model)
            sim.run(w.t_end, w.seed)
            assert np.array_equal(sim.counts(), ref), w.name
    sims = [rd.Simulation(w.mesh, w.model, w.counts) for w in ws]
    try:
        rd.rdsplit_ensemble_run([s.h for s in sims], [w.t_end for w in ws], [w.seed for w in ws])
        for w, s, ref in zip(ws, sims, refs):
            assert np.array_equal(s.counts(), ref), (w.name, "engine")
    finally:
        for s in sims:
            s.close()
