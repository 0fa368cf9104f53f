"""Transfer rules on the GPU (Sec. II.C; Sec. III.B, Fig. 7).

1. Parity: under each comparison rule (first-order N(tau), half-step
   N(tau/2)) the CUDA path, dense and batched, gives exactly the oracle's
   counts under the same rule (tolerance 0).
2. The accuracy comparison of Fig. 7, on a synthetic stand-in for the
   paper's cylinder: a 4 um tube (2 x 2 x 40 Kuhn cells, 960 tets) with a
   constant zero-order influx into the tets of its two end layers, run from
   empty for ~1000 periods, 1024 realisations per rule through the batched
   engine.  The exact mean of the master equation (a linear system: the
   influx ODE) is the reference.  Each rule's sample mean profile along the
   tube must match that rule's own exact expectation under operator
   splitting, and the end-layer error of first-order splitting must exceed
   that of the method (the mean-occupancy rule), as the paper reports.
"""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I
from tests.laws import influx_ode_mean, influx_split_mean

pytestmark = pytest.mark.gpu

AVOGADRO = 6.02214076e23


@pytest.fixture(scope="module")
def rd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def _reaction_workloads():
    out = []
    m = I.cube(5, 1e-6, 0.2, 12)
    n = I.molecules(20e-6, 1e-18)
    out.append(I.Workload("abc_n5", m, I.abc_model(), I.place_by_volume(m, [n, n, n // 3], 4), 2e-3, 7))
    bar = I.kuhn_box(4, 4, 12, (0.2e-6, 0.2e-6, 0.6e-6), 0.2, 13)
    V = 0.2e-6 * 0.2e-6 * 0.6e-6
    f, b = I.molecules(5e-6, V), I.molecules(50e-6, V)
    out.append(I.Workload("bar_4x4x12", bar, I.bar_model(bar), I.place_by_volume(bar, [f, f, f, b, b, 0, 0, 0], 5),
                          1.2e-3, 9))
    w = I.serving_requests(64)[5].workload()
    w.t_end = min(w.t_end, 2e-3)
    out.append(w)
    return out


@pytest.mark.parametrize("rule", [1, 2])
def test_rules_bit_exact_dense_and_batched(rd, oracle, rule):
    ws = _reaction_workloads()
    refs = [oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed, rule=rule)[0] for w in ws]
    for w, ref in zip(ws, refs):
        with rd.Simulation(w.mesh, w.model, w.counts, rule=rule) as sim:
            sim.run(w.t_end, w.seed)
            assert np.array_equal(sim.counts(), ref), (w.name, rule)
    sims = [rd.Simulation(w.mesh, w.model, w.counts, rule=rule) for w in ws]
    try:
        rd.rdsplit_ensemble_run([s.h for s in sims], [w.t_end for w in ws], [w.seed for w in ws])
        for w, s, ref in zip(ws, sims, refs):
            assert np.array_equal(s.counts(), ref), (w.name, rule, "engine")
    finally:
        for s in sims:
            s.close()
    # the rule matters: the method's own rule gives other counts here
    base = oracle.run(ws[1].mesh, ws[1].model, ws[1].counts, ws[1].t_end, ws[1].seed)[0]
    assert not np.array_equal(base, refs[1])


def _tube(a_tau: float):
    L, w, nz, D = 4e-6, 0.2e-6, 40, 1e-12
    mesh = I.kuhn_box(2, 2, nz, (w, w, L), 0.2, 77)
    z = mesh.centroid[:, 2]
    ends = (z < L / nz) | (z > L - L / nz)
    model0 = I.diffusion_model(D)
    from oracle import oracle as O
    tau = O.tau(mesh, model0)
    vol_l = float(np.mean(mesh.vol[ends])) * 1e3
    k_in = a_tau / (tau * AVOGADRO * vol_l)          # M/s: a_tau molecules per period in a mean end tet
    model = I.Model(D=np.array([D]), lhs=np.zeros((1, 1), np.int32), rhs=np.ones((1, 1), np.int32),
                    k=np.array([k_in]), mask=ends[None, :].astype(np.uint8))
    a = np.where(ends, k_in * AVOGADRO * mesh.vol * 1e3, 0.0)   # molecules/s per tet
    bins = np.minimum((z / (L / nz)).astype(int), nz - 1)
    return mesh, model, tau, a, bins, nz, D


def test_tube_influx_first_order_error_exceeds_mean_rule(rd):
    import torch
    a_tau, periods, n_real, n_handles = 4.0, 1000, 1024, 256
    mesh, model, tau, a, bins, nz, D = _tube(a_tau)
    t_end = periods * tau
    ode = np.bincount(bins, influx_ode_mean(mesh, D, a, t_end), nz)
    expect = {c: np.bincount(bins, influx_split_mean(mesh, D, a, tau, periods, c), nz) for c in (0.5, 1.0)}
    zero = np.zeros((mesh.n_tets, 1), np.int32)
    stream = torch.cuda.current_stream()
    sims = [rd.Simulation(mesh, model, zero, stream=stream) for _ in range(n_handles)]
    prof = {}
    try:
        for rule in (0, 1, 2):
            rows = []
            for batch in range(n_real // n_handles):
                for s in sims:
                    rd.rdsplit_set_transfer_rule(s.h, rule)
                    s.set_counts(zero)
                    rd.rdsplit_set_time(s.h, 0.0, 0)
                seeds = [1 + batch * n_handles + i for i in range(n_handles)]
                rd.rdsplit_ensemble_run([s.h for s in sims], [t_end] * n_handles, seeds)
                for s in sims:
                    assert s.time[1] == periods
                    rows.append(np.bincount(bins, s.counts()[:, 0].astype(np.float64), nz))
            prof[rule] = np.array(rows)
    finally:
        for s in sims:
            s.close()
    ends = [0, nz - 1]
    err = {}
    for rule, c in ((0, 0.5), (1, 1.0), (2, 0.5)):
        mean = prof[rule].mean(0)
        se = prof[rule].std(0, ddof=1) / np.sqrt(n_real)
        z = (mean - expect[c]) / se
        # the sample mean is that rule's exact split-scheme expectation
        assert np.max(np.abs(z)) < 5.0, (rule, np.round(z, 2))
        err[rule] = (mean - ode)[ends].sum()
        se_end = np.sqrt((se[ends] ** 2).sum())
        print(f"rule {rule}: end-layer error vs the master equation {err[rule]:.1f} +- {se_end:.1f} "
              f"(expected {(expect[c] - ode)[ends].sum():.1f}); mean |error| per bin "
              f"{np.abs(mean - ode).mean():.2f}")
    # Fig. 7(c, d): first-order splitting is further from the exact mean
    assert abs(err[1]) > abs(err[0]) + 4 * np.sqrt(2) * se_end
    assert abs(err[1]) > abs(err[2]) + 4 * np.sqrt(2) * se_end
