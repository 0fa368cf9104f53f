"""Reactions with a doubled reactant (2A -> ...) on the GPU: the
'production and second-order degradation' model of Sec. III.B (Fig. 6), in
one tet (a single exact-SSA period) and on a small mesh with diffusion,
dense and batched, equal the oracle count for count (tolerance 0)."""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I
from tests.laws import one_tet_mesh
from tests.test_oracle_laws import production_dimer_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def test_dimer_decay_one_tet(rd, oracle):
    vol = 1e-19
    mesh = one_tet_mesh(vol)
    model = production_dimer_model(vol, 40.0, 3.0)
    c0 = np.array([[3]], np.int32)
    for seed in range(12):
        ref = oracle.run(mesh, model, c0, 0.4, seed)[0]
        with rd.Simulation(mesh, model, c0) as sim:
            sim.run(0.4, seed)
            assert np.array_equal(sim.counts(), ref), seed


def test_dimer_decay_with_diffusion_dense_and_batched(rd, oracle):
    m = I.cube(4, 1e-6, 0.2, 3)
    vol = float(m.vol.mean())
    model = production_dimer_model(vol, 2000.0, 50.0, D=0.5e-12)
    c0 = np.full((m.n_tets, 1), 4, np.int32)
    t_end, seed = 0.05, 11
    ref = oracle.run(m, model, c0, t_end, seed)[0]
    with rd.Simulation(m, model, c0) as sim:
        sim.run(t_end, seed)
        assert np.array_equal(sim.counts(), ref)
    with rd.Simulation(m, model, c0) as sim:
        rd.rdsplit_ensemble_run([sim.h], [t_end], [seed])
        assert np.array_equal(sim.counts(), ref)
