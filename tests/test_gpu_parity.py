"""GPU parity: the CUDA path through the C ABI against the serial oracle.

Counts are integers drawn from the same keyed random streams with the same
IEEE-754 binary64 arithmetic on both sides, so parity is bit-exact equality of
every count (tolerance 0).
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I
from tests.laws import one_tet_mesh, two_tet_mesh

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_runs.json")


@pytest.fixture(scope="module")
def rd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def gpu_run(rd, w, t_end=None, max_periods=None, tau_scale=None, mode=0, block=0):
    model = w.model
    if tau_scale is not None:
        model.tau_scale = tau_scale
    with rd.Simulation(w.mesh, model, w.counts) as sim:
        rd.rdsplit_set_period_kernel(sim.h, mode, block)
        if max_periods is not None:
            sim.run_periods(max_periods, w.seed)
        else:
            sim.run(w.t_end if t_end is None else t_end, w.seed)
        return sim.counts(), sim.time


def oracle_run(oracle, w, t_end=None, max_periods=None):
    if max_periods is not None:
        c, t, p = oracle.run(w.mesh, w.model, w.counts, np.inf, w.seed, max_periods=max_periods)
    else:
        c, t, p = oracle.run(w.mesh, w.model, w.counts, w.t_end if t_end is None else t_end, w.seed)
    return c, (t, p)


def assert_same(gpu, ora):
    assert gpu.shape == ora.shape
    bad = np.argwhere(gpu != ora)
    assert bad.size == 0, f"{len(bad)} counts differ, first at {bad[:5].tolist()}"


def test_diffusion_cube_3072_full_run(rd, oracle):
    w = I.config_diffusion_3072()
    g, (tg, pg) = gpu_run(rd, w)
    o, (to, po) = oracle_run(oracle, w)
    assert_same(g, o)
    assert tg == to and pg == po == 217


def _small_cases():
    cases = {}
    w = I.diffusion_cube(4, 1e-6, 0.2, 11, 6000, 0.0137, 3)          # binomial path, short last period
    cases["diffusion_n4_point_source"] = w
    m = I.cube(5, 1e-6, 0.2, 12)
    n = I.molecules(20e-6, 1e-18)
    cases["abc_n5_dense"] = I.Workload("abc_n5", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4),
                                       2e-3, 7)
    bar = I.kuhn_box(4, 4, 40, (0.2e-6, 0.2e-6, 2e-6), 0.2, 13)
    bm = I.bar_model(bar)
    V = 0.2e-6 * 0.2e-6 * 2e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    cases["bar_4x4x40_masked_influx"] = I.Workload("bar_small", bar, bm,
                                                   I.place_by_volume(bar, [f, f, f, b, b, 0, 0, 0], 5), 1.5e-3, 9)
    return cases


@pytest.mark.parametrize("mode, block", [(0, 0), (1, 256), (1, 64), (2, 256), (2, 96)])
@pytest.mark.parametrize("name", list(_small_cases().keys()))
def test_small_workloads_bit_exact(rd, oracle, name, mode, block):
    """One-pass and two-pass period kernels (any light-pass block size)
    give the oracle's counts."""
    w = _small_cases()[name]
    g, (tg, pg) = gpu_run(rd, w, mode=mode, block=block)
    o, (to, po) = oracle_run(oracle, w)
    assert pg == po and tg == to
    assert_same(g, o)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("rid", [1, 2, 5, 7, 8, 13])
def test_random_chemistries_bit_exact(rd, oracle, rid, mode):
    req = I.serving_requests(64)[rid]
    w = req.workload()
    w.t_end = min(w.t_end, 3e-3)
    g, _ = gpu_run(rd, w, mode=mode)
    o, _ = oracle_run(oracle, w)
    assert_same(g, o)


def test_tau_scale_and_ragged_sizes(rd, oracle):
    # T = 6 * 3^3 = 162 (one partial block), tau scaled down
    w = I.diffusion_cube(3, 1e-6, 0.2, 21, 37, 0.01, 5)
    w.model.tau_scale = 0.37
    g, _ = gpu_run(rd, w)
    o, _ = oracle_run(oracle, w)
    assert_same(g, o)


def test_single_tet_reactions_only(rd, oracle):
    """No face neighbours: tau is infinite and a run is one period of exact SSA."""
    vol = 1e-19
    m = one_tet_mesh(vol)
    nav = 6.02214076e23 * vol * 1e3
    model = I.Model(D=np.array([1e-12, 1e-12, 1e-12]), lhs=np.array([[1, 1, 0], [0, 0, 1]], np.int32),
                    rhs=np.array([[0, 0, 1], [1, 1, 0]], np.int32), k=np.array([0.5 * nav, 2.0]))
    for seed in range(20):
        w = I.Workload("one", m, model, np.array([[40, 30, 0]], np.int32), 0.7, seed)
        g, (tg, pg) = gpu_run(rd, w)
        o, (to, po) = oracle_run(oracle, w)
        assert_same(g, o)
        assert pg == po == 1


def test_two_tets_and_empty_state(rd, oracle):
    m = two_tet_mesh()
    w = I.Workload("two", m, I.diffusion_model(1e-12), np.array([[13], [0]], np.int32), 1.0, 3)
    g, _ = gpu_run(rd, w)
    o, _ = oracle_run(oracle, w)
    assert_same(g, o)
    w0 = I.config_diffusion_3072()
    w0.counts[:] = 0
    g, _ = gpu_run(rd, w0)
    assert np.all(g == 0)


@pytest.mark.parametrize("mode", [1, 2])
def test_reaction_diffusion_48k_prefix(rd, oracle, mode):
    w = I.config_reaction_diffusion_48k()
    g, (tg, pg) = gpu_run(rd, w, max_periods=120, mode=mode)
    o, (to, po) = oracle_run(oracle, w, max_periods=120)
    assert pg == po == 120
    assert_same(g, o)


def test_resume_equals_single_run(rd, oracle):
    """Counts, time and period index are the whole state: stopping on a
    period boundary, copying the counts to a fresh handle and continuing
    gives the same result as one run."""
    w = I.diffusion_cube(5, 1e-6, 0.2, 31, 900, 0.03, 17)
    with rd.Simulation(w.mesh, w.model, w.counts) as a:
        a.run_periods(23, w.seed)
        mid = a.counts()
        t, p = a.time
        with rd.Simulation(w.mesh, w.model, mid) as b:
            rd.rdsplit_set_time(b.h, t, p)
            b.run(w.t_end, w.seed)
            resumed = b.counts()
        a.run(w.t_end, w.seed)
        straight = a.counts()
    assert_same(resumed, straight)
    o, _ = oracle_run(oracle, w)
    assert_same(straight, o)


def test_seed_changes_result_and_repeats(rd):
    w = I.diffusion_cube(4, 1e-6, 0.2, 11, 500, 0.01, 3)
    a, _ = gpu_run(rd, w)
    b, _ = gpu_run(rd, w)
    w.seed = 4
    c, _ = gpu_run(rd, w)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_device_pointer_counts(rd, oracle):
    import torch
    w = I.diffusion_cube(4, 1e-6, 0.2, 11, 300, 0.01, 3)
    with rd.Simulation(w.mesh, w.model) as sim:
        x = torch.from_numpy(w.counts).cuda()
        rd.rdsplit_set_counts_device(sim.h, x)
        sim.run(w.t_end, w.seed)
        y = torch.empty_like(x)
        rd.rdsplit_get_counts_device(sim.h, y)
        torch.cuda.synchronize()
        o, _ = oracle_run(oracle, w)
        assert_same(y.cpu().numpy(), o)


def test_invalid_inputs_are_rejected(rd):
    m = I.cube(2)
    adj = m.adj.copy()
    u = next(x for x in range(1, m.n_tets) if 0 not in m.adj[x])
    adj[0, 0] = u                      # u does not point back to tet 0
    with pytest.raises(rd.RdsplitError) as e:
        rd.rdsplit_mesh_create(m.n_tets, adj, m.vol, m.area, m.dist)
    assert e.value.code == rd.RDSPLIT_EINVAL
    vol = m.vol.copy()
    vol[3] = -1.0
    with pytest.raises(rd.RdsplitError) as e:
        rd.rdsplit_mesh_create(m.n_tets, m.adj, vol, m.area, m.dist)
    assert e.value.code == rd.RDSPLIT_EINVAL
    h = rd.rdsplit_mesh_create(m.n_tets, m.adj, m.vol, m.area, m.dist)
    try:
        with pytest.raises(rd.RdsplitError) as e:
            rd.rdsplit_run(h, 1.0, 1)
        assert e.value.code == rd.RDSPLIT_ESTATE
        with pytest.raises(rd.RdsplitError):
            rd.rdsplit_set_model(h, 17, np.ones(17), 0, None, None, None)
        rd.rdsplit_set_model(h, 1, [1e-12], 0, None, None, None)
        c = np.zeros((m.n_tets, 1), np.int32)
        c[4] = -3
        with pytest.raises(rd.RdsplitError) as e:
            rd.rdsplit_set_counts(h, c)
        assert e.value.code == rd.RDSPLIT_EINVAL
    finally:
        rd.rdsplit_mesh_destroy(h)


def _golden():
    if not os.path.exists(GOLDEN):
        return {}
    return json.load(open(GOLDEN))


def _golden_workload(rec):
    kind, args = rec["kind"], rec["args"]
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


def _golden_cases():
    names = sorted(_golden().keys())
    # the automatic kernel form (one pass), and two passes on the bar and the
    # 48k-cube prefixes
    return [(n, 0) for n in names] + [("bar_20x20x1000@20", 2), ("reaction_diffusion_cube_48000@300", 2)]


@pytest.mark.parametrize("name, mode", _golden_cases())
def test_full_size_against_stored_oracle_runs(rd, name, mode):
    """Full-size workloads against the SHA-256 of the oracle's final counts
    (written by tests/golden/make_golden.py from the oracle alone)."""
    rec = _golden()[name]
    w = _golden_workload(rec)
    mp = rec["max_periods"]
    g, (t, p) = gpu_run(rd, w, max_periods=mp if mp >= 0 else None, mode=mode)
    assert p == rec["period"]
    assert [int(x) for x in g.sum(0)] == rec["totals"]
    assert hashlib.sha256(np.ascontiguousarray(g, dtype="<i4").tobytes()).hexdigest() == rec["sha256"]


@pytest.mark.parametrize("k", [1, 4])
def test_zeta_outliers_bit_exact(rd, oracle, k):
    """The outlier option (Sec. II.A): tau from the (k+1)-th fastest tet,
    equal to the oracle's, and the run equals the oracle's with the same
    option, dense and batched."""
    m = I.cube(5, 1e-6, 0.2, 12)
    n = I.molecules(20e-6, 1e-18)
    w = I.Workload("abc_n5", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4), 2e-3, 7)
    ref, t_ref, p_ref = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed, outliers=k)
    with rd.Simulation(w.mesh, w.model, w.counts) as sim:
        base_tau = sim.tau
        rd.rdsplit_set_zeta_outliers(sim.h, k)
        assert sim.tau == oracle.tau(w.mesh, w.model, outliers=k) > base_tau
        sim.run(w.t_end, w.seed)
        assert_same(sim.counts(), ref)
        assert sim.time == (t_ref, p_ref)
    with rd.Simulation(w.mesh, w.model, w.counts) as sim:
        rd.rdsplit_set_zeta_outliers(sim.h, k)
        rd.rdsplit_ensemble_run([sim.h], [w.t_end], [w.seed])
        assert_same(sim.counts(), ref)


def test_zeta_histogram(rd):
    """Fig. 1d diagnostic: the histogram of zeta over the tets matches the
    same quantity computed on the host from the mesh, and the outlier option
    moves k tets to zeta = 1."""
    m = I.cube(6, 1e-6, 0.2, 5)
    model = I.diffusion_model(1e-12)
    inner = m.adj >= 0
    g = np.where(inner, m.area / (m.vol[:, None] * np.where(inner, m.dist, 1.0)), 0.0)
    G = ((g[:, 0] + g[:, 1]) + g[:, 2]) + g[:, 3]
    with rd.Simulation(m, model) as sim:
        for k in (0, 6):
            if k:
                rd.rdsplit_set_zeta_outliers(sim.h, k)
            z = np.minimum(1.0, sim.tau * (1e-12 * G))
            counts, mean, mx = rd.rdsplit_zeta_histogram(sim.h, 20)
            ref = np.bincount(np.minimum((z * 20).astype(int), 19), minlength=20)
            assert counts.sum() == m.n_tets
            assert np.abs(counts - ref).max() <= 1
            assert abs(mean - z.mean()) < 1e-12 and abs(mx - z.max()) <= 1e-15
            assert (z >= 1.0).sum() >= k and counts[-1] >= k
