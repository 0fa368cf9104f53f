"""Lockstep engine (batched ensemble and continuous batching) against the
serial oracle: every simulation in the engine must end with exactly the
counts the oracle gives it alone (tolerance 0), however it is mixed."""
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
    out = []
    for i, n in enumerate([3, 5, 4, 6, 2]):
        w = I.diffusion_cube(n, 1e-6, 0.2, 40 + i, 6000 if i % 2 == 0 else 7, 0.004 + 0.002 * i, 11 + i)
        out.append(w)
    m = I.cube(4, 1e-6, 0.2, 12)
    nmol = I.molecules(20e-6, 1e-18)
    out.append(I.Workload("abc_n4", m, I.abc_model(), I.place_by_volume(m, [nmol, nmol, nmol // 3], 4), 2e-3, 7))
    bar = I.kuhn_box(3, 3, 12, (0.15e-6, 0.15e-6, 0.6e-6), 0.2, 13)
    V = 0.15e-6 * 0.15e-6 * 0.6e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    out.append(I.Workload("bar_3x3x12", bar, I.bar_model(bar), I.place_by_volume(bar, [f, f, f, b, b, 0, 0, 0], 5),
                          1.0e-3, 9))
    for rid in (2, 7, 13):
        w = I.serving_requests(64)[rid].workload()
        w.t_end = min(w.t_end, 2e-3)
        out.append(w)
    return out


def _oracle(oracle, w):
    return oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)[0]


def test_ensemble_matches_oracle_per_instance(rd, oracle):
    ws = _workloads()
    sims = [rd.Simulation(w.mesh, w.model, w.counts) for w in ws]
    try:
        rd.rdsplit_ensemble_run([s.h for s in sims], [w.t_end for w in ws], [w.seed for w in ws])
        for w, s in zip(ws, sims):
            got = s.counts()
            assert np.array_equal(got, _oracle(oracle, w)), w.name
            t, p = s.time
            assert t == w.t_end
    finally:
        for s in sims:
            s.close()


def test_continuous_batching_mix_is_invisible(rd, oracle):
    """Simulations joining at different global steps, with others finishing
    and their slots reused, each end exactly as when run alone."""
    ws = _workloads()
    e = rd.rdsplit_engine_create(3, sum(w.mesh.n_tets for w in ws))
    sims = {}
    try:
        pending = list(range(len(ws)))
        done = []
        steps = 0
        while pending or sims:
            while pending and len(sims) < 3:
                i = pending.pop(0)
                s = rd.Simulation(ws[i].mesh, ws[i].model, ws[i].counts)
                slot = rd.rdsplit_engine_add(e, s.h, ws[i].t_end, ws[i].seed)
                sims[slot] = (i, s)
            rd.rdsplit_engine_step(e, 7 + (steps % 5))
            steps += 1
            for slot in rd.rdsplit_engine_poll(e):
                i, s = sims.pop(slot)
                done.append((i, s.counts()))
                s.close()
        assert len(done) == len(ws)
        for i, got in done:
            assert np.array_equal(got, _oracle(oracle, ws[i])), ws[i].name
    finally:
        rd.rdsplit_engine_destroy(e)
        for _, s in sims.values():
            s.close()


def test_engine_admission_limits(rd):
    w = _workloads()[0]
    e = rd.rdsplit_engine_create(1, w.mesh.n_tets)
    a = rd.Simulation(w.mesh, w.model, w.counts)
    b = rd.Simulation(w.mesh, w.model, w.counts)
    try:
        rd.rdsplit_engine_add(e, a.h, w.t_end, 1)
        with pytest.raises(rd.RdsplitError) as err:
            rd.rdsplit_engine_add(e, b.h, w.t_end, 1)
        assert err.value.code == rd.RDSPLIT_ENOMEM
        rd.rdsplit_engine_step(e, 1 << 30)
        assert rd.rdsplit_engine_active(e) == (0, 0)
        assert rd.rdsplit_engine_poll(e) == [0]
    finally:
        rd.rdsplit_engine_destroy(e)
        a.close()
        b.close()


def test_engine_matches_dense_path_after_resume(rd):
    """A handle advanced first with rdsplit_run_periods and then finished in
    the engine equals one rdsplit_run."""
    w = I.diffusion_cube(5, 1e-6, 0.2, 31, 900, 0.03, 17)
    with rd.Simulation(w.mesh, w.model, w.counts) as a:
        a.run(w.t_end, w.seed)
        ref = a.counts()
    with rd.Simulation(w.mesh, w.model, w.counts) as b:
        b.run_periods(23, w.seed)
        rd.rdsplit_ensemble_run([b.h], [w.t_end], [w.seed])
        assert np.array_equal(b.counts(), ref)


@pytest.fixture(scope="module")
def oracle_results(oracle):
    return [_oracle(oracle, w) for w in _workloads()]


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("in_flight", [1, 3, 0])
def test_every_cluster_shape_matches_oracle(rd, oracle_results, cluster, in_flight):
    """The engine's result does not depend on how many CTAs share a
    simulation or how many simulations run at once (0: as many as fit)."""
    ws = _workloads()
    sims = [rd.Simulation(w.mesh, w.model, w.counts) for w in ws]
    e = rd.rdsplit_engine_create(len(ws), sum(w.mesh.n_tets for w in ws))
    try:
        rd.rdsplit_engine_set_concurrency(e, in_flight, cluster)
        for w, s in zip(ws, sims):
            rd.rdsplit_engine_add(e, s.h, w.t_end, w.seed)
        rd.rdsplit_engine_step(e, 1 << 30)
        assert sorted(rd.rdsplit_engine_poll(e, 64)) == list(range(len(ws)))
        for w, s, ref in zip(ws, sims, oracle_results):
            assert np.array_equal(s.counts(), ref), (w.name, cluster, in_flight)
    finally:
        rd.rdsplit_engine_destroy(e)
        for s in sims:
            s.close()


def test_cluster_sizes_other_than_1_2_4_8_are_rejected(rd):
    e = rd.rdsplit_engine_create(1, 1000)
    try:
        for bad in (0, 3, 16):
            with pytest.raises(rd.RdsplitError) as err:
                rd.rdsplit_engine_set_concurrency(e, 0, bad)
            assert err.value.code == rd.RDSPLIT_EINVAL
        with pytest.raises(rd.RdsplitError):
            rd.rdsplit_engine_set_concurrency(e, -1, 2)
        rd.rdsplit_engine_set_concurrency(e, 0, 8)
        assert rd.rdsplit_engine_active(e) == (0, 0)
    finally:
        rd.rdsplit_engine_destroy(e)


def _stored_full_runs():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_runs.json")
    recs = {k: v for k, v in json.load(open(path)).items()
            if v["kind"] in ("ensemble", "request") and v["max_periods"] < 0}
    ws, names = [], []
    for name, rec in sorted(recs.items()):
        a = rec["args"]
        ws.append(I.ensemble_instance(a["i"], a["n"]) if rec["kind"] == "ensemble"
                  else I.serving_requests(64)[a["rid"]].workload())
        names.append(name)
    return recs, ws, names


def _check_stored(recs, names, sims):
    import hashlib
    for name, s in zip(names, sims):
        rec = recs[name]
        g = s.counts()
        t, p = s.time
        assert p == rec["period"], name
        assert [int(x) for x in g.sum(0)] == rec["totals"], name
        assert hashlib.sha256(np.ascontiguousarray(g, dtype="<i4").tobytes()).hexdigest() == rec["sha256"], name


def test_full_size_ensemble_and_requests_in_one_launch(rd):
    """Every stored full-size oracle run of an ensemble instance or a serving
    request (tests/golden/oracle_runs.json, written from the oracle alone),
    all advanced together by one persistent engine launch in the default
    launch configuration, ends with the oracle's counts (SHA-256 of the final
    counts, period index and per-species totals)."""
    recs, ws, names = _stored_full_runs()
    assert len(recs) >= 60
    sims = [rd.Simulation(w.mesh, w.model, w.counts) for w in ws]
    try:
        rd.rdsplit_ensemble_run([s.h for s in sims], [w.t_end for w in ws], [w.seed for w in ws])
        _check_stored(recs, names, sims)
    finally:
        for s in sims:
            s.close()


def test_full_size_in_equal_cost_slices(rd):
    """The same stored runs advanced in many launches whose slices give each
    simulation about the same work (rdsplit_engine_set_slice_work: large
    meshes advance fewer periods per launch), as continuous batching does:
    identical results."""
    recs, ws, names = _stored_full_runs()
    sims = [rd.Simulation(w.mesh, w.model, w.counts) for w in ws]
    e = rd.rdsplit_engine_create(len(ws), sum(w.mesh.n_tets for w in ws))
    try:
        rd.rdsplit_engine_set_slice_work(e, 30_000_000)
        for w, s in zip(ws, sims):
            rd.rdsplit_engine_add(e, s.h, w.t_end, w.seed)
        steps = 0
        while rd.rdsplit_engine_active(e)[0] > 0:
            rd.rdsplit_engine_step(e, 700)
            rd.rdsplit_engine_poll(e)
            steps += 1
        assert steps > 10
        _check_stored(recs, names, sims)
    finally:
        rd.rdsplit_engine_destroy(e)
        for s in sims:
            s.close()


def test_deferred_queue_overflow_and_resume(rd, oracle):
    """A dense reaction workload (most tets have a reaction event in every
    period, so most tets take the deferred full step): with one CTA per
    simulation each warp defers far more than its 64-entry queue per period,
    so the light pass stops and resumes many times."""
    m = I.cube(8, 1e-6, 0.2, 21)
    n = I.molecules(400e-6, 1e-18)
    w = I.Workload("abc_dense", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 4], 6), 2e-3, 5)
    ref = _oracle(oracle, w)
    for cluster in (1, 4, 8):
        with rd.Simulation(w.mesh, w.model, w.counts) as s:
            e = rd.rdsplit_engine_create(1, m.n_tets)
            try:
                rd.rdsplit_engine_set_concurrency(e, 1, cluster)
                rd.rdsplit_engine_add(e, s.h, w.t_end, w.seed)
                rd.rdsplit_engine_step(e, 1 << 30)
            finally:
                rd.rdsplit_engine_destroy(e)
            assert np.array_equal(s.counts(), ref), cluster


def _line_of_three():
    """Tets A - B - C; A and C have half B's volume, so zeta = 1 in them (every
    molecule leaves each period) and 1/2 in B."""
    from paper_1512_03126_gb300.inputs import Mesh
    adj = np.array([[1, -1, -1, -1], [0, 2, -1, -1], [1, -1, -1, -1]], np.int32)
    area = np.zeros((3, 4))
    dist = np.zeros((3, 4))
    area[0, 0] = area[1, 0] = area[1, 1] = area[2, 0] = 1e-13
    dist[0, 0] = dist[1, 0] = dist[1, 1] = dist[2, 0] = 2e-7
    return Mesh(adj=adj, vol=np.array([1e-19, 4e-19, 1e-19]), area=area, dist=dist,
                centroid=np.array([[0, 0, 0], [2e-7, 0, 0], [4e-7, 0, 0]], np.float64), shape=(), size=(1, 1, 1))


@pytest.mark.parametrize("cluster", [1, 2])
def test_count_overflow_is_reported_like_the_oracle(rd, oracle, cluster):
    """A count pushed past 2^31-1 by the transfers: A and C each hold 1.2e9
    molecules and send all of them to B in the first period.  The oracle,
    the period kernel and the batched engine (whose adds are fire-and-forget:
    the wrapped count is caught when read back) all report the overflow;
    with 1.0e9 each none does, and the three agree."""
    m = _line_of_three()
    model = I.diffusion_model(1e-12)
    for each, overflows in ((1_200_000_000, True), (1_000_000_000, False)):
        c0 = np.array([[each], [0], [each]], np.int32)
        if overflows:
            with pytest.raises(oracle.OracleError):
                oracle.run(m, model, c0, np.inf, 3, max_periods=2)
        else:
            ref, _, _ = oracle.run(m, model, c0, np.inf, 3, max_periods=2)
        with rd.Simulation(m, model, c0) as s:
            if overflows:
                with pytest.raises(rd.RdsplitError) as e:
                    s.run_periods(2, 3)
                assert e.value.code == rd.RDSPLIT_EOVERFLOW
            else:
                s.run_periods(2, 3)
                assert np.array_equal(s.counts(), ref)
        with rd.Simulation(m, model, c0) as s:
            tau = s.tau
            e = rd.rdsplit_engine_create(1, 3)
            try:
                rd.rdsplit_engine_set_concurrency(e, 1, cluster)
                rd.rdsplit_engine_add(e, s.h, 2 * tau, 3)
                if overflows:
                    with pytest.raises(rd.RdsplitError) as err:
                        rd.rdsplit_engine_step(e, 1 << 30)
                    assert err.value.code == rd.RDSPLIT_EOVERFLOW
                else:
                    rd.rdsplit_engine_step(e, 1 << 30)
                    assert np.array_equal(s.counts(), ref)
            finally:
                rd.rdsplit_engine_destroy(e)


def test_adding_with_t_end_in_the_past_keeps_the_state(rd):
    """A simulation added with t_end at or before its current time runs no
    period and keeps its time, period index and counts, as rdsplit_run does
    for such a t_end."""
    w = I.diffusion_cube(4, 1e-6, 0.2, 11, 300, 0.004, 3)
    with rd.Simulation(w.mesh, w.model, w.counts) as a, rd.Simulation(w.mesh, w.model, w.counts) as b:
        a.run(w.t_end, w.seed)
        b.run(w.t_end, w.seed)
        ta, pa = a.time
        ca = a.counts()
        a.run(0.5 * w.t_end, w.seed)                 # dense path: a no-op
        e = rd.rdsplit_engine_create(1, w.mesh.n_tets)
        try:
            rd.rdsplit_engine_add(e, b.h, 0.5 * w.t_end, w.seed)
            rd.rdsplit_engine_step(e, 10)
            assert rd.rdsplit_engine_active(e)[0] == 0
        finally:
            rd.rdsplit_engine_destroy(e)
        assert a.time == (ta, pa) == b.time
        assert np.array_equal(a.counts(), ca) and np.array_equal(b.counts(), ca)
