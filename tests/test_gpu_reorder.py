"""Space-filling-curve storage order (RDSPLIT_REORDER_SFC): a mesh whose tets
are numbered at random runs with the same counts, in the caller's order,
whether the library keeps that numbering or stores the tets along a Morton
curve of their centroids; both equal the oracle (tolerance 0), through the
period kernel and through the batched engine."""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    import torch
    assert torch.cuda.is_available()
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def _shuffled_cases():
    out = []
    m, old = I.shuffle_mesh(I.cube(6, 1e-6, 0.2, 41), 7)
    n = I.molecules(20e-6, 1e-18)
    out.append(I.Workload("abc_n6_shuffled", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 8), 1.5e-3, 3))
    bar = I.kuhn_box(4, 4, 40, (0.2e-6, 0.2e-6, 2e-6), 0.2, 13)
    bm = I.bar_model(bar)
    bar_s, old = I.shuffle_mesh(bar, 9)
    bm.mask = np.ascontiguousarray(bm.mask[:, old])
    V = 0.2e-6 * 0.2e-6 * 2e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    out.append(I.Workload("bar_small_shuffled", bar_s, bm, I.place_by_volume(bar_s, [f, f, f, b, b, 0, 0, 0], 5),
                          1.0e-3, 9))
    w = I.ensemble_instance(5, 12, 0.01)
    ms, _ = I.shuffle_mesh(w.mesh, 11)
    out.append(I.Workload("point_source_shuffled", ms, w.model, I.point_source(ms, 1, 0, 6000), 0.01, 5))
    return out


@pytest.mark.parametrize("k", range(3))
def test_reorder_keeps_results(rd, oracle, k):
    w = _shuffled_cases()[k]
    ref, _, _ = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
    got = {}
    for reorder in (False, True):
        with rd.Simulation(w.mesh, w.model, w.counts, reorder=reorder) as sim:
            order = rd.rdsplit_get_order(sim.h)
            assert sorted(order) == list(range(w.mesh.n_tets))
            if reorder:
                # stored neighbours are close in space: consecutive stored
                # tets are much nearer each other than in the random numbering
                c = w.mesh.centroid
                near = np.linalg.norm(np.diff(c[order], axis=0), axis=1).mean()
                far = np.linalg.norm(np.diff(c, axis=0), axis=1).mean()
                assert near < 0.5 * far
            else:
                assert np.array_equal(order, np.arange(w.mesh.n_tets))
            sim.run(w.t_end, w.seed)
            got[reorder] = sim.counts()
        with rd.Simulation(w.mesh, w.model, w.counts, reorder=reorder) as sim:
            rd.rdsplit_ensemble_run([sim.h], [w.t_end], [w.seed])
            assert np.array_equal(sim.counts(), ref), (w.name, reorder, "engine")
    assert np.array_equal(got[False], ref)
    assert np.array_equal(got[True], ref)


def test_reorder_needs_centroids(rd):
    m = I.cube(2)
    with pytest.raises(rd.RdsplitError) as e:
        rd.rdsplit_mesh_create(m.n_tets, m.adj, m.vol, m.area, m.dist, rd.RDSPLIT_REORDER_SFC)
    assert e.value.code == rd.RDSPLIT_EINVAL
    c = m.centroid.copy()
    c[3, 1] = np.nan
    with pytest.raises(rd.RdsplitError):
        rd.rdsplit_mesh_create_ex(m.n_tets, m.adj, m.vol, m.area, m.dist, c, rd.RDSPLIT_REORDER_SFC)
