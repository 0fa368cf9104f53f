// Per-tet device functions of one operator-splitting period (Algorithm 1 of
// arXiv:1512.03126, Step 2 and Step 3), shared by the period kernels.
#pragma once
#include "rd_device.cuh"
#include "rd_internal.h"

namespace rdk {

constexpr int kEventCap = 1 << 22;   // SSA events per tet and period
constexpr double kAvogadro = 6.02214076e23;

// Transfer probability over a period of length tau_k (Eq. 1 and the text
// after it): zeta = tau_k * D * G, at most 1.
__device__ __forceinline__ double zeta_of(double tau_k, double D, double Gt) {
    double z = tau_k * (D * Gt);
    return z > 1.0 ? 1.0 : z;
}

// Incoming molecules of species s for tet t: what each neighbour sent through
// the shared face in the previous period.
__device__ __forceinline__ int64_t incoming(const int32_t* __restrict__ op, int4 sr) {
    int64_t n = 0;
    if (sr.x >= 0) n += __ldg(op + sr.x);
    if (sr.y >= 0) n += __ldg(op + sr.y);
    if (sr.z >= 0) n += __ldg(op + sr.z);
    if (sr.w >= 0) n += __ldg(op + sr.w);
    return n;
}

// Reaction phase of one tet (Algorithm 1, Step 2 and 2.1): Gillespie's
// direct method over [0, tau_k); the first event at or past tau_k is
// discarded.  Before a species' count changes, its occupancy integral
// advances by N * (t_event - t_last).
__device__ __forceinline__ void react_tet(const DevMesh& m, const ModelParams& mp, int t, uint32_t period,
                                          double tau_k, uint64_t seed, int64_t* N, double* occ, double* tl,
                                          uint32_t& touched, uint32_t* err) {
    double avv = kAvogadro * (m.vol[t] * 1000.0);
    uint32_t on = mp.has_mask ? m.mask[t] : 0xffffffffu;
    rdd::Stream st(seed, (uint32_t)t, period, rdd::kPurposeReaction, 0);
    double tc = 0.0;
    int events = 0;
    for (;;) {
        double a[kMaxR];
        double a0 = 0.0;
        for (int r = 0; r < mp.R; ++r) {
            double ar = 0.0;
            if ((on >> r) & 1u) {
                int64_t h = 1;
                for (int s = 0; s < mp.S; ++s) {
                    int nu = mp.lhs[r][s];
                    if (nu == 1) h = h * N[s];
                    else if (nu == 2) h = h * (N[s] * (N[s] - 1) / 2);
                }
                if (h != 0) {
                    double kr = mp.k[r];
                    int o = mp.order[r];
                    double c = o == 0 ? kr * avv : (o == 1 ? kr : kr / avv);
                    ar = c * (double)h;
                }
            }
            a[r] = ar;
            a0 = a0 + ar;
        }
        if (!(a0 > 0.0)) break;
        double u1 = st.u01_open0();
        double tn = tc + (-rdd::own_log(u1)) / a0;
        if (tn >= tau_k) break;
        double target = st.u01() * a0;
        int mu = -1;
        double cum = 0.0;
        for (int r = 0; r < mp.R; ++r) {
            cum = cum + a[r];
            if (target < cum) { mu = r; break; }
        }
        if (mu < 0)
            for (int r = mp.R - 1; r >= 0; --r)
                if (a[r] > 0.0) { mu = r; break; }
        for (int s = 0; s < mp.S; ++s) {
            int dn = mp.delta[mu][s];
            if (dn != 0) {
                occ[s] = occ[s] + (double)N[s] * (tn - tl[s]);
                tl[s] = tn;
                touched |= 1u << s;
                N[s] += dn;
            }
        }
        tc = tn;
        if (++events >= kEventCap) { atomicOr(err, kErrEventCap); break; }
    }
    for (int s = 0; s < mp.S; ++s)
        if ((touched >> s) & 1u) occ[s] = occ[s] + (double)N[s] * (tau_k - tl[s]);
}

// Diffusion of one species out of one tet (Algorithm 1, Step 3; Eq. 2-3;
// Sec. II.B): N* from the occupancy (stochastic rounding of N-bar when the
// count changed during the period, else N), n = min(Binomial(N*, zeta), N),
// split over the faces by conditional binomials; below N* = 10 the same law
// one molecule at a time against the cumulative thresholds.
__device__ __forceinline__ int4 diffuse(const DevMesh& m, int t, int s, double Dsp, uint32_t period, double tau_k,
                                        uint64_t seed, int64_t Nt, bool touched, double occ, uint4 C) {
    int4 o = make_int4(0, 0, 0, 0);
    double Gt = m.G[t];
    double z = zeta_of(tau_k, Dsp, Gt);
    if (!(z > 0.0) || Nt <= 0) return o;
    int64_t Nstar = Nt;
    if (touched) {
        rdd::Stream rs(seed, (uint32_t)t, period, rdd::kPurposeRounding, (uint32_t)s);
        double nbar = occ / tau_k;
        double fl = floor(nbar);
        double frac = nbar - fl;
        Nstar = (int64_t)fl + (rs.u01() < frac ? 1 : 0);
    }
    if (Nstar <= 0) return o;
    rdd::Stream ds(seed, (uint32_t)t, period, rdd::kPurposeDiffusion, (uint32_t)s);
    if (Nstar < 10) {
        int64_t moved = 0;
        for (int64_t i = 0; i < Nstar; ++i) {
            if (moved == Nt) break;
            uint32_t u = ds.u32();
            if (rdd::below(u, C.x)) { o.x += 1; ++moved; }
            else if (rdd::below(u, C.y)) { o.y += 1; ++moved; }
            else if (rdd::below(u, C.z)) { o.z += 1; ++moved; }
            else if (rdd::below(u, C.w)) { o.w += 1; ++moved; }
        }
        return o;
    }
    int64_t n = rdd::binomial(Nstar, z, ds);
    if (n > Nt) n = Nt;
    if (n == 0) return o;
    double g[4];
    for (int f = 0; f < 4; ++f) g[f] = m.g[4 * t + f];
    double suf[4];
    double acc = 0.0;
    for (int f = 3; f >= 0; --f) { acc = g[f] + acc; suf[f] = acc; }
    int last = -1;
    for (int f = 0; f < 4; ++f)
        if (g[f] > 0.0) last = f;
    int64_t rest = n;
    int64_t nf[4] = {0, 0, 0, 0};
    for (int f = 0; f < 4; ++f) {
        if (!(g[f] > 0.0)) continue;
        if (f == last) { nf[f] = rest; break; }
        int64_t x = rdd::binomial(rest, g[f] / suf[f], ds);
        nf[f] = x;
        rest -= x;
    }
    o = make_int4((int)nf[0], (int)nf[1], (int)nf[2], (int)nf[3]);
    return o;
}

}  // namespace rdk
