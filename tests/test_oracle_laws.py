"""Pins of the serial oracle (Algorithm 1) against what the mathematics and
the paper fix: conservation, the exact law of pure diffusion under operator
splitting, exact reaction laws, the mean-corrected transfer of Eq. 2-3, the
continuum spreading rate, and a brute-force exact spatial SSA."""
import math

import numpy as np
import pytest
from scipy.stats import binom

from paper_1512_03126_gb300 import inputs as I
from tests.laws import (binomial_of_shifted_poisson, birth_death_ABC, chi2_pvalue, mean_rule_influx_law,
                        one_period_matrix, one_tet_mesh, production_dimer_decay, two_tet_mesh)


def _src(counts):
    return int(np.nonzero(counts.sum(1))[0][0])


def test_conservation_and_sign(oracle):
    """Pure diffusion moves molecules between tets and never creates or
    destroys them; counts stay >= 0 (Sec. II.A, transfer-based diffusion)."""
    w = I.config_diffusion_3072()
    c = w.counts.copy()
    t, per = 0.0, 0
    for _ in range(5):
        c, t, per = oracle.run(w.mesh, w.model, c, w.t_end, w.seed, t0=t, period0=per, max_periods=20)
        assert c.sum() == 6000 and c.min() >= 0
    assert per == 100


def test_period_rule_and_alignment(oracle):
    """tau = 1 / max(D_s * sum_f A/(V dist)) (Algorithm 1, precompute); the last
    period is shortened to land on t_end (Step 1)."""
    w = I.config_diffusion_3072()
    tau = oracle.tau(w.mesh, w.model)
    g = np.where(w.mesh.adj >= 0, w.mesh.area / (w.mesh.vol[:, None] * np.where(w.mesh.dist > 0, w.mesh.dist, 1)), 0)
    assert tau == pytest.approx(1.0 / (1e-12 * g.sum(1).max()), rel=1e-12)
    # 4.623e-4 s on the 1 um 8^3 Kuhn cube with D = 1e-12 m^2/s
    assert tau == pytest.approx(4.623e-4, rel=1e-3)
    c, t, per = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)
    assert t == w.t_end and per == math.ceil(w.t_end / tau)


@pytest.mark.parametrize("n0", [6, 300, 6000])
def test_exact_law_of_pure_diffusion(oracle, n0):
    """With N-bar = N each molecule independently takes one step of the
    period matrix M per period (leave with probability zeta = tau*d, direction
    multinomial by face weight), so the count in tet u after k periods is
    Binomial(N0, (e_src M^k)_u) and the pooled positions are multinomial.
    n0 = 6 and 300 exercise the one-draw-per-molecule path, n0 = 6000 (above
    the 4096 cut) the binomial + conditional-binomial path in its first
    period."""
    m = I.cube(2, 0.5e-6, 0.2, 7)
    model = I.diffusion_model(1e-12)
    c0 = np.zeros((m.n_tets, 1), np.int32)
    src = 17
    c0[src, 0] = n0
    tau = oracle.tau(m, model)
    k = 6
    p = np.linalg.matrix_power(one_period_matrix(m, 1e-12, tau), k)[src]
    seeds = 3000 if n0 < 1000 else 600
    finals = np.stack([oracle.run(m, model, c0, np.inf, s, max_periods=k)[0][:, 0] for s in range(seeds)])
    assert np.all(finals.sum(1) == n0)
    pooled = finals.sum(0)
    assert chi2_pvalue(pooled, p) > 1e-4
    u = int(np.argmax(p))
    obs = np.bincount(finals[:, u], minlength=n0 + 1)
    assert chi2_pvalue(obs, binom.pmf(np.arange(n0 + 1), n0, p[u])) > 1e-4


def test_zeta_one_empties_the_fastest_tet(oracle):
    """On a regular mesh zeta = 1 in the fastest tets (Sec. II.A): every
    molecule there leaves in one period, in both sampler paths."""
    m = I.cube(3, 1e-6, 0.0, 0)
    model = I.diffusion_model(1e-12)
    g = np.where(m.adj >= 0, m.area / (m.vol[:, None] * np.where(m.dist > 0, m.dist, 1)), 0).sum(1)
    fast = int(np.nonzero(g == g.max())[0][0])
    for n0 in (7, 500, 5000):
        c0 = np.zeros((m.n_tets, 1), np.int32)
        c0[fast, 0] = n0
        for s in range(20):
            c, _, _ = oracle.run(m, model, c0, np.inf, s, max_periods=1)
            assert c[fast, 0] == 0 and c.sum() == n0


def test_first_order_decay_is_exactly_binomial(oracle):
    """Per-tet SSA is exact for A -> 0 and diffusion neither creates nor
    destroys molecules, so survivors ~ Binomial(N0, exp(-k t)) exactly."""
    m = I.cube(2, 0.5e-6, 0.2, 7)
    kdec = 20.0
    model = I.Model(D=np.array([1e-12]), lhs=np.array([[1]], np.int32), rhs=np.array([[0]], np.int32),
                    k=np.array([kdec]))
    c0 = np.zeros((m.n_tets, 1), np.int32)
    c0[5, 0] = 200
    t_end = math.log(2.0) / kdec
    tot = np.array([oracle.run(m, model, c0, t_end, s)[0].sum() for s in range(3000)])
    obs = np.bincount(tot, minlength=201)
    assert chi2_pvalue(obs, binom.pmf(np.arange(201), 200, math.exp(-kdec * t_end))) > 1e-4


def _abc(k1_pair_rate, k2, vol):
    """A + B <-> C with the given per-pair forward rate (1/s) in a tet of
    volume ``vol``, plus a diffusing spectator Z that fixes tau."""
    nav = 6.02214076e23 * vol * 1e3
    lhs = np.array([[1, 1, 0, 0], [0, 0, 1, 0]], np.int32)
    rhs = np.array([[0, 0, 1, 0], [1, 1, 0, 0]], np.int32)
    return I.Model(D=np.array([0.0, 0.0, 0.0, 1e-12]), lhs=lhs, rhs=rhs,
                   k=np.array([k1_pair_rate * nav, k2]), tau_scale=0.1)


@pytest.mark.parametrize("two_tets", [False, True])
def test_reversible_binding_matches_master_equation(oracle, two_tets):
    """A + B <-> C in one tet: the law of C(t) is the birth-death chain of the
    chemical master equation.  With one tet there is a single period; with
    two tets and a diffusing spectator the SSA restarts every period, which
    must not change the law (memoryless events)."""
    vol = 1e-19
    model = _abc(0.5, 2.0, vol)
    mesh = two_tet_mesh((vol, vol)) if two_tets else one_tet_mesh(vol)
    c0 = np.zeros((mesh.n_tets, 4), np.int32)
    c0[0, 0], c0[0, 1] = 8, 6
    t_end = 0.3
    if two_tets:
        assert oracle.tau(mesh, model) < t_end / 5
    C = np.array([oracle.run(mesh, model, c0, t_end, s)[0][0, 2] for s in range(4000)])
    law = birth_death_ABC(8, 6, 0.5, 2.0, 0, t_end)
    assert chi2_pvalue(np.bincount(C, minlength=law.size), law) > 1e-4


def production_dimer_model(vol: float, lam: float, c2: float, D: float = 0.0):
    """0 -> A at lam molecules/s in a tet of volume vol, and 2A -> 0 at c2
    per pair (the 'production and second-order degradation' model of
    Sec. III.B, Fig. 6), in SI rate constants."""
    nav = 6.02214076e23 * vol * 1e3
    return I.Model(D=np.array([D]), lhs=np.array([[0], [2]], np.int32), rhs=np.array([[1], [0]], np.int32),
                   k=np.array([lam / nav, c2 * nav]))


def test_production_and_dimer_decay_matches_master_equation(oracle):
    """Fig. 6's model in one tet: 0 -> A and 2A -> 0.  The law of A(t) is
    the master equation's, which pins the propensity of a reaction with a
    doubled reactant, c N (N - 1) / 2."""
    vol = 1e-19
    lam, c2, t_end = 40.0, 3.0, 0.4
    mesh = one_tet_mesh(vol)
    model = production_dimer_model(vol, lam, c2)
    A = np.array([oracle.run(mesh, model, np.array([[3]], np.int32), t_end, s)[0][0, 0] for s in range(4000)])
    law = production_dimer_decay(lam, c2, 3, t_end, 60)
    assert law[-5:].sum() < 1e-12
    assert chi2_pvalue(np.bincount(A, minlength=law.size), law) > 1e-4


def test_mean_corrected_transfer(oracle):
    """Eq. 2-3: the number leaving a tet over a period is drawn from the mean
    occupancy N-bar during the period, not N at its end.  With a zero-order
    influx of rate a into a tet holding N0, E[N-bar] = N0 + a tau / 2, so
    E[n] = zeta (N0 + a tau / 2); first-order splitting would give
    zeta (N0 + a tau)."""
    vol = 1e-19
    mesh = two_tet_mesh((vol, vol))
    D = 1e-12
    zeta = 0.5
    model0 = I.diffusion_model(D)
    model0.tau_scale = zeta
    tau = oracle.tau(mesh, model0)
    a_tau = 20.0
    k_in = a_tau / (tau * 6.02214076e23 * vol * 1e3)
    mask = np.array([[1, 0]], np.uint8)
    model = I.Model(D=np.array([D]), lhs=np.zeros((1, 1), np.int32), rhs=np.ones((1, 1), np.int32),
                    k=np.array([k_in]), mask=mask, tau_scale=zeta)
    c0 = np.array([[5], [0]], np.int32)
    n = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1)[0][1, 0] for s in range(20000)])
    expect = zeta * (5 + a_tau / 2)
    se = n.std() / math.sqrt(n.size)
    assert abs(n.mean() - expect) < 4 * se
    assert abs(n.mean() - zeta * (5 + a_tau)) > 20 * se


def _influx_two_tets(a_tau: float, zeta: float):
    """Two tets; tet 0 holds 5 molecules and has a zero-order influx of
    a_tau molecules per period (mean); tau set so that zeta = tau * d."""
    vol = 1e-19
    mesh = two_tet_mesh((vol, vol))
    D = 1e-12
    model0 = I.diffusion_model(D)
    model0.tau_scale = zeta
    tau = oracle_tau(mesh, model0)
    k_in = a_tau / (tau * 6.02214076e23 * vol * 1e3)
    mask = np.array([[1, 0]], np.uint8)
    model = I.Model(D=np.array([D]), lhs=np.zeros((1, 1), np.int32), rhs=np.ones((1, 1), np.int32),
                    k=np.array([k_in]), mask=mask, tau_scale=zeta)
    return mesh, model, np.array([[5], [0]], np.int32)


def oracle_tau(mesh, model):
    from oracle import oracle as O
    return O.tau(mesh, model)


@pytest.mark.parametrize("rule", [1, 2])
def test_comparison_rules_exact_laws(oracle, rule):
    """The comparison transfer rules of Sec. II.C and III.B.  With a Poisson
    influx (a tau per period) into a tet holding N0 = 5 and no other
    reaction, the count at time s of the period is N0 + Poisson(a s), so the
    number sent to the other tet in one period is exactly
    Binomial(N0 + Poisson(a tau), zeta) under first-order splitting (N at
    tau) and Binomial(N0 + Poisson(a tau / 2), zeta) under the half-step
    reading (N at tau / 2).  The method's rule (N-bar) has the second one's
    mean but not its law (the random part of N-bar has variance a tau / 3,
    that of N(tau / 2) a tau / 2), and the test checks that the law tells
    them apart."""
    zeta, a_tau = 0.5, 20.0
    mesh, model, c0 = _influx_two_tets(a_tau, zeta)
    n = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1, rule=rule)[0][1, 0]
                  for s in range(20000)])
    lam = a_tau if rule == 1 else a_tau / 2
    law = binomial_of_shifted_poisson(5, lam, zeta, int(n.max()) + 20)
    assert chi2_pvalue(np.bincount(n, minlength=law.size), law) > 1e-4
    if rule == 2:
        mean_rule = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1)[0][1, 0]
                              for s in range(20000)])
        assert chi2_pvalue(np.bincount(mean_rule, minlength=law.size), law) < 1e-6


@pytest.mark.parametrize("n0, a_tau, zeta, seeds", [(5, 20.0, 0.5, 20000), (0, 2.0, 1.0, 40000)])
def test_mean_rule_exact_law(oracle, n0, a_tau, zeta, seeds):
    """The law, not only the mean, of the method's transfer (Eq. 3 with the
    unbiased stochastic rounding of reading 4): with a Poisson influx the
    occupancy mean is N0 plus a sum of uniforms, and the sent count has the
    closed-form law of laws.mean_rule_influx_law (chi-square).  With zeta = 1
    every counted molecule leaves, so the second case sees N* itself, where
    a rounding to the nearest integer instead of the stochastic one shows."""
    mesh, model, c0 = _influx_two_tets(a_tau, zeta)
    c0[0, 0] = n0
    n = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1)[0][1, 0] for s in range(seeds)])
    law = mean_rule_influx_law(n0, a_tau, zeta, int(n.max()) + 20)
    assert chi2_pvalue(np.bincount(n, minlength=law.size), law) > 1e-4
    if zeta < 1.0:
        other = binomial_of_shifted_poisson(n0, a_tau / 2, zeta, law.size - 1)
        assert chi2_pvalue(np.bincount(n, minlength=law.size), other) < 1e-6


def test_transfer_is_capped_by_the_molecules_present(oracle):
    """Reading 5: n = min(Binomial(N*, zeta), N(tau_k)).  Under a first-order
    decay N-bar exceeds the survivors N(tau_k) (counts only fall), so with
    zeta = 1 the cap binds: exactly the survivors leave.  The tet ends empty
    and its neighbour holds Binomial(40, e^{-k tau}) molecules."""
    vol = 1e-19
    mesh = two_tet_mesh((vol, vol))
    model0 = I.diffusion_model(1e-12)
    model0.tau_scale = 1.0
    tau = oracle.tau(mesh, model0)
    k = 2.0 / tau
    model = I.Model(D=np.array([1e-12]), lhs=np.ones((1, 1), np.int32), rhs=np.zeros((1, 1), np.int32),
                    k=np.array([k]), tau_scale=1.0)
    c0 = np.array([[40], [0]], np.int32)
    got = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1)[0][:, 0] for s in range(3000)])
    assert np.all(got[:, 0] == 0)
    law = binom.pmf(np.arange(41), 40, math.exp(-2.0))
    assert chi2_pvalue(np.bincount(got[:, 1], minlength=41), law) > 1e-4


def _decay_transfer_law(n0: int, k_tau: float, zeta: float, cap_first: bool, samples: int, seed: int):
    """Monte Carlo (numpy, independent of the oracle) of the molecules sent in
    one period by a tet holding n0 molecules that decay at rate k, with
    transfer probability zeta: each molecule lives Exp(k); N-bar is the
    summed lifetime inside the period over tau; N* its unbiased stochastic
    rounding; N(tau) the survivors.  cap_first = False: n =
    min(Binomial(N*, zeta), N(tau)) (reading 5); True: n = Binomial(min(N*,
    N(tau)), zeta).  Returns the pmf of n over 0..n0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    life = rng.exponential(1.0 / k_tau, size=(samples, n0))       # in units of tau
    nbar = np.minimum(life, 1.0).sum(1)
    surv = (life >= 1.0).sum(1)
    fl = np.floor(nbar)
    nstar = (fl + (rng.random(samples) < nbar - fl)).astype(np.int64)
    if cap_first:
        n = rng.binomial(np.minimum(nstar, surv), zeta)
    else:
        n = np.minimum(rng.binomial(nstar, zeta), surv)
    return np.bincount(n, minlength=n0 + 1)[: n0 + 1] / samples


def test_transfer_cap_law_below_zeta_one(oracle):
    """Reading 5 at zeta = 1/2, where it differs from capping N* before the
    draw: under a first-order decay N-bar exceeds the survivors N(tau_k), and
    the method sends n = min(Binomial(N*, zeta), N(tau_k)).  The oracle's
    count sent to the neighbour in one period follows that law (chi-square
    against an independent Monte Carlo of the decay), and not the law of
    Binomial(min(N*, N(tau_k)), zeta)."""
    vol = 1e-19
    mesh = two_tet_mesh((vol, vol))
    zeta = 0.5
    model0 = I.diffusion_model(1e-12)
    model0.tau_scale = zeta
    tau = oracle.tau(mesh, model0)
    k_tau = 1.2
    model = I.Model(D=np.array([1e-12]), lhs=np.ones((1, 1), np.int32), rhs=np.zeros((1, 1), np.int32),
                    k=np.array([k_tau / tau]), tau_scale=zeta)
    n0 = 30
    c0 = np.array([[n0], [0]], np.int32)
    got = np.array([oracle.run(mesh, model, c0, np.inf, s, max_periods=1)[0][:, 0] for s in range(8000)])
    sent = np.bincount(got[:, 1], minlength=n0 + 1)
    law = _decay_transfer_law(n0, k_tau, zeta, False, 400_000, 5)
    other = _decay_transfer_law(n0, k_tau, zeta, True, 400_000, 6)
    assert chi2_pvalue(sent, law) > 1e-4
    assert chi2_pvalue(sent, other) < 1e-6


def test_rules_agree_without_reactions(oracle):
    """Without reactions N-bar = N(tau/2) = N(tau): the three rules give the
    same counts, draw for draw."""
    w = I.diffusion_cube(4, 1e-6, 0.2, 11, 600, 0.004, 3)
    base = oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed)[0]
    for rule in (1, 2):
        assert np.array_equal(oracle.run(w.mesh, w.model, w.counts, w.t_end, w.seed, rule=rule)[0], base)


def _rates_numpy(mesh, D):
    """Per-tet rates d_t = D * (g0 + g1 + g2 + g3), g_f = A / (V dist), in the
    same floating-point operations as the method's setup (Sec. II.A)."""
    inner = mesh.adj >= 0
    g = np.where(inner, mesh.area / (mesh.vol[:, None] * np.where(inner, mesh.dist, 1.0)), 0.0)
    G = ((g[:, 0] + g[:, 1]) + g[:, 2]) + g[:, 3]
    return D * G


@pytest.mark.parametrize("k", [0, 1, 5])
def test_outlier_option_takes_tau_from_the_next_tet(oracle, k):
    """Sec. II.A: leaving the k tets with the highest zeta out of the choice
    of tau gives tau = tau_scale / d_(k+1), the (k+1)-th largest per-tet rate."""
    m = I.cube(4, 1e-6, 0.2, 31)
    model = I.diffusion_model(1e-12)
    model.tau_scale = 0.8
    d = np.sort(_rates_numpy(m, 1e-12))[::-1]
    assert oracle.tau(m, model, outliers=k) == 0.8 / d[k]


def test_outlier_tets_have_zeta_one(oracle):
    """With the three fastest tets left out of the choice of tau, the second
    fastest has tau * d > 1, so zeta = 1 there: every molecule leaves it in
    one period (and some stay without the option, where zeta = d_2/d_1 < 1)."""
    m = I.cube(4, 1e-6, 0.2, 31)
    model = I.diffusion_model(1e-12)
    d = _rates_numpy(m, 1e-12)
    order = np.argsort(-d)
    assert d[order[1]] < d[order[0]] and d[order[1]] > d[order[3]]
    c0 = np.zeros((m.n_tets, 1), np.int32)
    c0[order[1], 0] = 1000
    left = oracle.run(m, model, c0, np.inf, 3, max_periods=1, outliers=3)[0]
    assert left[order[1], 0] == 0 and left.sum() == 1000
    kept = oracle.run(m, model, c0, np.inf, 3, max_periods=1)[0]
    assert kept[order[1], 0] > 0


def test_point_source_spreads_at_6Dt(oracle):
    """Volume diffusion speed (Sec. III.A): from a point source the mean
    squared displacement grows as 6 D t in 3-D (before the walls matter)."""
    m = I.cube(12, 3e-6, 0.2, 9)
    model = I.diffusion_model(1e-12)
    c0 = I.point_source(m, 1, 0, 2000)
    src = _src(c0)
    t_end = 0.055
    c, t, _ = oracle.run(m, model, c0, t_end, 5)
    msd = (c[:, 0][:, None] * (m.centroid - m.centroid[src]) ** 2).sum() / 2000
    assert 0.9 < msd / (6e-12 * t_end) < 1.1


def _moment_se(x: np.ndarray):
    """Per-column sample mean and variance of x [n][...] with their standard
    errors (the variance's from the sample fourth central moment)."""
    n = x.shape[0]
    m = x.mean(0)
    d = x - m
    v = (d ** 2).sum(0) / (n - 1)
    m4 = (d ** 4).mean(0)
    se_m = np.sqrt(v / n)
    se_v = np.sqrt(np.maximum(m4 - v ** 2 * (n - 3) / (n - 1), 0.0) / n)
    return m, v, se_m, se_v


def test_agrees_with_exact_spatial_ssa(oracle):
    """Brute force (Sec. I and III: the exact ISSA is the reference of the
    method's accuracy): on a 48-tet jittered box with diffusion and
    A + B <-> C, the per-tet means and variances of every species under
    operator splitting (tau scaled to 0.1, so that the O(tau) splitting bias
    stays below the resolution) match those of the exact whole-mesh SSA
    within 4 standard errors, over 10^4 seeds of each."""
    m = I.kuhn_box(2, 2, 2, (1e-6, 1e-6, 1e-6), 0.2, 17)
    assert m.n_tets == 48
    nav = 6.02214076e23 * m.vol.mean() * 1e3
    lhs = np.array([[1, 1, 0], [0, 0, 1]], np.int32)
    rhs = np.array([[0, 0, 1], [1, 1, 0]], np.int32)
    model = I.Model(D=np.array([1e-12, 0.5e-12, 0.2e-12]), lhs=lhs, rhs=rhs,
                    k=np.array([2.0 * nav, 5.0]), tau_scale=0.1)
    c0 = np.zeros((m.n_tets, 3), np.int32)
    c0[0] = (20, 15, 0)
    c0[47] = (0, 10, 5)
    t_end = 0.03
    n = 10_000
    os_ = np.stack([oracle.run(m, model, c0, t_end, s)[0] for s in range(n)]).astype(float)
    ex = np.stack([oracle.issa_run(m, model, c0, t_end, 10**6 + s) for s in range(n)]).astype(float)
    mo, vo, smo, svo = _moment_se(os_)
    me, ve, sme, sve = _moment_se(ex)
    tiny = 1e-12
    assert np.all(np.abs(mo - me) <= 4.0 * np.sqrt(smo ** 2 + sme ** 2) + tiny)
    assert np.all(np.abs(vo - ve) <= 4.0 * np.sqrt(svo ** 2 + sve ** 2) + tiny)
    # both are genuinely stochastic, moved mass away from the sources, and
    # reacted (C formed from A + B)
    assert ex[:, 0, 0].mean() < 20 and os_[:, 0, 0].mean() < 20
    assert (ex[:, :, 2].sum(1) != 5).mean() > 0.5
    assert np.all(ve[ve > 0.05] > 0)
