"""Validation foils of Sec. II.A (Fig. 2): the discrete-mean count and the
net-flux transfer, which the paper shows to lose spatial noise, against the
method's binomial gross transfer.

Pins of the foils themselves (closed forms), then the Fig. 2(d) analogue on
a jittered 384-tet cube: the stationary per-tet variance of a closed pure-
diffusion system is that of the multinomial law with p_t = V_t / V (each
molecule independent, detailed balance V_t d_tu = V_u d_ut also holds for the
split scheme), and the method reproduces it while the foils fall short.
"""
import numpy as np
import pytest

from paper_1512_03126_gb300 import inputs as I
from tests.laws import two_tet_mesh


def test_mean_n_foil_moves_the_rounded_mean(oracle):
    """Discrete mean (Fig. 2(b)): with two tets, n = floor(zeta N + 1/2)
    molecules cross in one period, for every seed."""
    m = two_tet_mesh()
    model = I.diffusion_model(1e-12)
    model.tau_scale = 0.37                     # zeta = 0.37 in both tets (equal volumes)
    for n0, seed in ((10, 1), (11, 2), (250, 3)):
        c0 = np.array([[n0], [0]], np.int32)
        got = oracle.run_foil(m, model, c0, np.inf, seed, oracle.FOIL_MEAN_N, max_periods=1)[0]
        assert got[1, 0] == int(np.floor(0.37 * n0 + 0.5)) and got.sum() == n0


def test_net_foil_moves_nothing_between_equal_tets(oracle):
    """Net flux (Fig. 2(c)): two equal tets with equal counts exchange
    nothing; from an empty neighbour the count sent is Binomial(N, zeta)."""
    m = two_tet_mesh()
    model = I.diffusion_model(1e-12)
    model.tau_scale = 0.5
    c0 = np.array([[40], [40]], np.int32)
    for seed in range(20):
        assert np.array_equal(oracle.run_foil(m, model, c0, np.inf, seed, oracle.FOIL_NET, max_periods=1)[0], c0)
    c1 = np.array([[200], [0]], np.int32)
    sent = np.array([oracle.run_foil(m, model, c1, np.inf, s, oracle.FOIL_NET, max_periods=1)[0][1, 0]
                     for s in range(4000)])
    assert abs(sent.mean() - 100.0) < 4 * np.sqrt(50.0 / sent.size)
    assert abs(sent.var() - 50.0) < 5.0


def _variance_ratio(oracle, density: int, foil: int) -> float:
    m = I.cube(4, 1e-6, 0.2, 8)
    model = I.diffusion_model(1e-12)
    vol = m.vol / m.vol.sum()
    n_tot = density * m.n_tets
    c = I.place_by_volume(m, [n_tot], 3)
    t, p = 0.0, 0
    samples = []
    for k in range(1100):
        if foil:
            c, t, p = oracle.run_foil(m, model, c, np.inf, 17, foil, t0=t, period0=p, max_periods=4)
        else:
            c, t, p = oracle.run(m, model, c, np.inf, 17, t0=t, period0=p, max_periods=4)
        if k >= 100:
            samples.append(c[:, 0].copy())
    x = np.array(samples, np.float64)
    expected = n_tot * vol * (1 - vol)
    return float(np.mean(x.var(0) / expected))


@pytest.mark.parametrize("density", [1, 10])
def test_spatial_noise_binomial_keeps_it_foils_lose_it(oracle, density):
    """Fig. 2(d): the method's per-tet stationary variance matches the exact
    multinomial law; the net-flux foil loses most of it (the paper: ~60% left
    at one molecule per tet, ~20% at ten) and the discrete mean loses some."""
    method = _variance_ratio(oracle, density, 0)
    net = _variance_ratio(oracle, density, oracle.FOIL_NET)
    mean_n = _variance_ratio(oracle, density, oracle.FOIL_MEAN_N)
    print(f"density {density}: variance / exact  method {method:.3f}  net {net:.3f}  mean-n {mean_n:.3f}")
    assert 0.9 < method < 1.1
    assert net < (0.8 if density == 1 else 0.4)
    assert mean_n < method - 0.05
