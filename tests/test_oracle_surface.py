"""Surface diffusion (Sec. III.A, Fig. 5(c, d): transfer between surface
triangles) through the same method and the same arrays: a triangle's area
takes the place of the tet volume, an edge's length that of a face area, and
the fourth neighbour slot is empty, so the hop rate across an edge is
D L / (A d).  Pins of the oracle on triangulated sheets."""
import numpy as np
import pytest
from scipy.stats import binom

from paper_1512_03126_gb300 import inputs as I
from tests.laws import chi2_pvalue, one_period_matrix


def test_sheet_is_a_valid_surface_mesh():
    m = I.triangle_sheet(8, 6, (1e-6, 0.75e-6), 0.2, 3)
    assert m.n_tets == 96 and abs(m.vol.sum() - 0.75e-12) < 1e-24
    assert np.all(m.adj[:, 3] == -1)
    for t in range(m.n_tets):
        for f in range(3):
            u = m.adj[t, f]
            if u >= 0:
                assert (m.adj[u] == t).sum() == 1
    assert (m.adj[:, :3] < 0).sum() == 2 * (8 + 6)    # edges on the rectangle's border


@pytest.mark.parametrize("n0", [300, 6000])
def test_exact_law_of_surface_diffusion(oracle, n0):
    """As in volume: each molecule independently takes one step of the
    period matrix per period, so counts after k periods are binomial and the
    pooled positions multinomial (n0 = 300: one draw per molecule; 6000: the
    binomial path in the first period)."""
    m = I.triangle_sheet(4, 4, (0.4e-6, 0.4e-6), 0.2, 5)
    model = I.diffusion_model(1e-12)
    c0 = np.zeros((m.n_tets, 1), np.int32)
    src = 13
    c0[src, 0] = n0
    tau = oracle.tau(m, model)
    k = 5
    p = np.linalg.matrix_power(one_period_matrix(m, 1e-12, tau), k)[src]
    seeds = 2000 if n0 < 1000 else 500
    finals = np.stack([oracle.run(m, model, c0, np.inf, s, max_periods=k)[0][:, 0] for s in range(seeds)])
    assert np.all(finals.sum(1) == n0)
    assert chi2_pvalue(finals.sum(0), p) > 1e-4
    u = int(np.argmax(p))
    obs = np.bincount(finals[:, u], minlength=n0 + 1)
    assert chi2_pvalue(obs, binom.pmf(np.arange(n0 + 1), n0, p[u])) > 1e-4


def test_point_source_spreads_at_4Dt_on_a_surface(oracle):
    """Surface diffusion speed (Fig. 5(c)): from a point source the mean
    squared displacement grows as 4 D t in 2-D (before the edges matter)."""
    m = I.triangle_sheet(40, 40, (4e-6, 4e-6), 0.2, 9)
    model = I.diffusion_model(1e-12)
    c0 = I.point_source(m, 1, 0, 3000, where=(2e-6, 2e-6, 0.0))
    src = int(np.argmax(c0[:, 0]))
    t_end = 0.08
    c, t, _ = oracle.run(m, model, c0, t_end, 5)
    msd = (c[:, 0][:, None] * (m.centroid - m.centroid[src]) ** 2).sum() / 3000
    assert 0.9 < msd / (4e-12 * t_end) < 1.1
