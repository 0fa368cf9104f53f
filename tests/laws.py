"""Exact laws used to pin the oracle (test helpers, numpy/scipy only).

Nothing here calls the oracle or the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm


def face_rates(mesh, D: float) -> np.ndarray:
    """Per-molecule hop rate t -> adj[t][f]: D * A_tf / (V_t * dist_tf)
    (the rate definition of the workload; 0 on the boundary)."""
    g = np.zeros_like(mesh.area)
    inner = mesh.adj >= 0
    g[inner] = mesh.area[inner] / (mesh.vol[:, None] * mesh.dist)[inner]
    return D * g


def one_period_matrix(mesh, D: float, tau_k: float) -> np.ndarray:
    """Transition matrix of one molecule over one period of pure diffusion:
    it leaves t through face f with probability tau_k * rate_tf (Eq. 1 text:
    the transfer probability over a period is zeta = tau * d; the direction
    is multinomial with weights proportional to the face rates)."""
    T = mesh.n_tets
    rate = face_rates(mesh, D)
    M = np.zeros((T, T))
    for t in range(T):
        for f in range(4):
            u = mesh.adj[t, f]
            if u >= 0:
                M[t, u] += tau_k * rate[t, f]
        M[t, t] = 1.0 - M[t].sum()
    return M


def birth_death_ABC(a0: int, b0: int, c_fwd: float, c_bwd: float, C0: int, t: float) -> np.ndarray:
    """Law of C(t) for A+B <-> C in one well-mixed volume with A+C=a0,
    B+C=b0 conserved: a birth-death chain with birth rate
    c_fwd*(a0-C)(b0-C) and death rate c_bwd*C, solved by a matrix
    exponential of its generator."""
    n = min(a0, b0) + 1
    Q = np.zeros((n, n))
    for c in range(n):
        up = c_fwd * (a0 - c) * (b0 - c)
        dn = c_bwd * c
        if c + 1 < n:
            Q[c, c + 1] = up
        if c > 0:
            Q[c, c - 1] = dn
        Q[c, c] = -(Q[c].sum())
    p0 = np.zeros(n)
    p0[C0] = 1.0
    return p0 @ expm(Q * t)


def chi2_pvalue(observed: np.ndarray, expected_p: np.ndarray, min_expected: float = 5.0) -> float:
    """Pearson chi-square goodness of fit with bins pooled so every expected
    count is at least ``min_expected``."""
    from scipy.stats import chi2
    n = observed.sum()
    e = expected_p * n
    obs_b, exp_b = [], []
    o_acc = e_acc = 0.0
    for o, x in zip(observed, e):
        o_acc += o
        e_acc += x
        if e_acc >= min_expected:
            obs_b.append(o_acc)
            exp_b.append(e_acc)
            o_acc = e_acc = 0.0
    if e_acc > 0 and exp_b:
        obs_b[-1] += o_acc
        exp_b[-1] += e_acc
    obs_b = np.array(obs_b)
    exp_b = np.array(exp_b)
    stat = ((obs_b - exp_b) ** 2 / exp_b).sum()
    dof = max(len(obs_b) - 1, 1)
    return float(chi2.sf(stat, dof))


def two_tet_mesh(vol=(1e-19, 1e-19), area=1e-13, dist=2e-7):
    """Two tets sharing face 0, all other faces on the boundary."""
    from paper_1512_03126_gb300.inputs import Mesh
    adj = np.array([[1, -1, -1, -1], [0, -1, -1, -1]], np.int32)
    a = np.zeros((2, 4))
    a[:, 0] = area
    d = np.zeros((2, 4))
    d[:, 0] = dist
    return Mesh(adj=adj, vol=np.array(vol, np.float64), area=a, dist=d,
                centroid=np.array([[0, 0, 0], [dist, 0, 0]], np.float64), shape=(), size=(1, 1, 1))


def one_tet_mesh(vol=1e-19):
    from paper_1512_03126_gb300.inputs import Mesh
    return Mesh(adj=np.full((1, 4), -1, np.int32), vol=np.array([vol]), area=np.full((1, 4), 1e-13),
                dist=np.zeros((1, 4)), centroid=np.zeros((1, 3)), shape=(), size=(1, 1, 1))


def binomial_of_shifted_poisson(n0: int, lam: float, p: float, kmax: int) -> np.ndarray:
    """pmf over k = 0..kmax of Binomial(n0 + M, p) with M ~ Poisson(lam)."""
    out = np.zeros(kmax + 1)
    mmax = int(lam + 12 * math.sqrt(lam) + 30)
    for m in range(mmax + 1):
        wm = math.exp(-lam + m * math.log(lam) - math.lgamma(m + 1)) if lam > 0 else float(m == 0)
        n = n0 + m
        for k in range(min(n, kmax) + 1):
            out[k] += wm * math.exp(math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1)
                                    + k * math.log(p) + (n - k) * math.log1p(-p))
    return out


def hop_generator(mesh, D: float) -> np.ndarray:
    """K with dm/dt = K m for the mean counts of pure diffusion in continuous
    time (the reaction-diffusion master equation's mean; K[u, t] = rate of a
    molecule's hop t -> u, K[t, t] = -(its total hop rate))."""
    T = mesh.n_tets
    rate = face_rates(mesh, D)
    K = np.zeros((T, T))
    for t in range(T):
        for f in range(4):
            u = mesh.adj[t, f]
            if u >= 0:
                K[u, t] += rate[t, f]
        K[t, t] -= rate[t].sum()
    return K


def influx_ode_mean(mesh, D: float, a: np.ndarray, t: float) -> np.ndarray:
    """Exact mean counts at time t from empty, under a constant influx a
    [molecules/s per tet] and diffusion: m(t) = int_0^t exp(K s) a ds (the
    master equation of a linear system has these means exactly)."""
    T = mesh.n_tets
    aug = np.zeros((T + 1, T + 1))
    aug[:T, :T] = hop_generator(mesh, D)
    aug[:T, T] = a
    return expm(aug * t)[:T, T]


def influx_split_mean(mesh, D: float, a: np.ndarray, tau: float, periods: int, c: float) -> np.ndarray:
    """Exact mean counts after `periods` operator-split periods from empty,
    under a constant influx a and pure diffusion, when the diffusion draw of
    a period uses a count whose mean is m + c a tau (m the count at the start
    of the period): c = 1/2 for the mean occupancy and for the count at
    mid-period, c = 1 for the count at the end (Sec. II.C).  Each molecule
    counted leaves t through face f with probability tau * rate_tf."""
    rate = face_rates(mesh, D)
    T = mesh.n_tets
    zeta = tau * rate.sum(1)
    W = np.zeros((T, T))
    for t in range(T):
        d = rate[t].sum()
        for f in range(4):
            u = mesh.adj[t, f]
            if u >= 0 and d > 0:
                W[u, t] += rate[t, f] / d
    m = np.zeros(T)
    for _ in range(periods):
        out = zeta * (m + c * a * tau)
        m = m + a * tau - out + W @ out
    return m


def production_dimer_decay(lam: float, c2: float, n0: int, t: float, n_max: int) -> np.ndarray:
    """Law of A(t) for 0 -> A (rate lam) and 2A -> 0 (rate c2 per unordered
    pair, so c2 * n (n - 1) / 2 in total) in one well-mixed volume, from
    A(0) = n0, on states 0..n_max (n_max well above where the law has mass):
    the chemical master equation solved by a matrix exponential."""
    n = n_max + 1
    Q = np.zeros((n, n))
    for a in range(n):
        if a + 1 < n:
            Q[a, a + 1] = lam
        if a >= 2:
            Q[a, a - 2] = c2 * a * (a - 1) / 2.0
        Q[a, a] = -(Q[a].sum())
    p0 = np.zeros(n)
    p0[n0] = 1.0
    return p0 @ expm(Q * t)


def irwin_hall_density_at_integer(n: int, x: int) -> float:
    """Density of the sum of n independent Uniform(0, 1) at the integer x,
    f_n(x) = sum_{k <= x} (-1)^k C(n, k) (x - k)^(n-1) / (n-1)!, evaluated in
    exact integer arithmetic (the alternating sum cancels badly in floats)."""
    if n < 1 or x <= 0 or x >= n:
        return 0.0
    num = sum((-1) ** k * math.comb(n, k) * (x - k) ** (n - 1) for k in range(0, x + 1))
    return num / math.factorial(n - 1)


def mean_rule_influx_law(n0: int, lam: float, zeta: float, kmax: int) -> np.ndarray:
    """Exact law of the count sent in one period under the mean-occupancy
    rule (Eq. 3 with unbiased stochastic rounding), for a tet holding n0 with
    a Poisson influx of mean lam over the period and one neighbour (all of
    zeta towards it), nothing else reacting.  Given m arrivals at uniform
    times, N-bar = n0 + S with S a sum of m uniforms; rounding gives
    N* = n0 + j with probability E[max(0, 1 - |S - j|)], which is the
    Irwin-Hall(m + 2) density at j + 1 (S plus the difference of two
    uniforms); then n ~ Binomial(N*, zeta)."""
    out = np.zeros(kmax + 1)
    mmax = int(lam + 12 * math.sqrt(lam) + 30)
    for m in range(mmax + 1):
        wm = math.exp(-lam + m * math.log(lam) - math.lgamma(m + 1))
        for j in range(0, m + 1):
            pj = 1.0 if m == 0 and j == 0 else irwin_hall_density_at_integer(m + 2, j + 1)
            if pj == 0.0:
                continue
            n = n0 + j
            if zeta >= 1.0:                       # every counted molecule leaves
                if n <= kmax:
                    out[n] += wm * pj
                continue
            k = np.arange(0, min(n, kmax) + 1)
            lg = np.array([math.lgamma(n + 1) - math.lgamma(i + 1) - math.lgamma(n - i + 1) for i in k])
            out[: k.size] += wm * pj * np.exp(lg + k * math.log(zeta) + (n - k) * math.log1p(-zeta))
    return out
