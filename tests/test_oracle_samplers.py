"""Pins of the oracle's samplers against exact laws (Sec. II.A-B)."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.stats import binom

from tests.laws import chi2_pvalue


@pytest.mark.parametrize("n,p", [
    (1, 0.3), (7, 0.5), (30, 0.2),          # inversion
    (100, 0.5), (6000, 0.37), (200, 0.93),  # BTRS, BTRS with p > 1/2
    (50, 0.999), (1000, 0.004),             # flipped inversion, small mean at large n
])
def test_binomial_exact_pmf(oracle, n, p):
    draws = oracle.binomial_many(n, p, 100000, seed=11)
    assert draws.min() >= 0 and draws.max() <= n
    obs = np.bincount(draws, minlength=n + 1)
    assert chi2_pvalue(obs, binom.pmf(np.arange(n + 1), n, p)) > 1e-4


def test_binomial_degenerate(oracle):
    assert np.all(oracle.binomial_many(0, 0.5, 10) == 0)
    assert np.all(oracle.binomial_many(17, 0.0, 10) == 0)
    assert np.all(oracle.binomial_many(17, 1.0, 10) == 17)


def test_paper_transfer_example(oracle):
    """Sec. II.C: with 10,000 molecules and 10% transferring per update,
    about 0.1 x 10,000 = 1,000 molecules move at each update."""
    d = oracle.binomial_many(10000, 0.1, 20000, seed=3)
    assert abs(d.mean() - 1000.0) < 4 * math.sqrt(10000 * 0.1 * 0.9 / d.size)


def test_threshold_is_floor_of_scaled_probability(oracle):
    rng = np.random.default_rng(5)
    for y in list(rng.uniform(0, 1, 2000)) + [0.0, 2.0**-32, 0.5, 1 - 2.0**-31]:
        exact = math.floor(Fraction(y) * 2**32)
        got = oracle.threshold(y)
        if exact >= 2**32 - 1:
            assert got == 0xFFFFFFFF
        else:
            assert got == exact
    assert oracle.threshold(1.0) == 0xFFFFFFFF
    assert oracle.threshold(1 - 2.0**-33) == 0xFFFFFFFF
