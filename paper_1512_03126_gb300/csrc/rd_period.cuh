// Per-tet device functions of one operator-splitting period (Algorithm 1 of
// arXiv:1512.03126, Step 2 and Step 3), shared by the period kernels.
#pragma once
#include "rd_device.cuh"
#include "rd_internal.h"

namespace rdk {

constexpr int kEventCap = 1 << 22;   // SSA events per tet and period
// Below this N* the diffusion draw is one uniform per molecule (the paper's
// per-molecule form, Sec. II.B); at or above it, Binomial + conditional
// binomials in double precision.
constexpr int64_t kMoleculeCut = 4096;
// From this N* up to kMoleculeCut, a warp draws the molecules of one tet
// together (untouched species only).
constexpr int32_t kWarpSplitMin = 10;
constexpr double kAvogadro = 6.02214076e23;

// Transfer probability over a period of length tau_k (Eq. 1 and the text
// after it): zeta = tau_k * D * G, at most 1.
__device__ __forceinline__ double zeta_of(double tau_k, double D, double Gt) {
    double z = tau_k * (D * Gt);
    return z > 1.0 ? 1.0 : z;
}

// Molecules that arrived in tet t during the previous period, added to n[s]
// for every species: the sum of t's four inbox slots (Sp = inbox_stride(S)
// ints each, 16-byte aligned as a whole), read with 16-byte loads.
template <int SA>
__device__ __forceinline__ void add_inbox(const int32_t* __restrict__ in, int64_t t, int S, int Sp, int64_t* n) {
    const int4* p = reinterpret_cast<const int4*>(in + t * 4 * Sp);
    if (SA == 1 || Sp == 1) {
        const int4 v = __ldg(p);
        n[0] += (int64_t)v.x + v.y + v.z + v.w;
        return;
    }
    if (SA == 2 || Sp == 2) {
        const int4 a = __ldg(p), b = __ldg(p + 1);
        n[0] += (int64_t)a.x + a.z + b.x + b.z;
        if (SA > 1) n[1] += (int64_t)a.y + a.w + b.y + b.w;
        return;
    }
    const int q4 = Sp >> 2;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int q = 0; q < (SA + 3) / 4; ++q) {
            if (q >= q4) break;
            const int4 v = __ldg(p + f * q4 + q);
            const int vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int sp = 4 * q + k;
                if (sp < SA && sp < S) n[sp < SA ? sp : 0] += vals[k];
            }
        }
    }
}

__device__ __forceinline__ int face_of(const int4& v, int f) {
    return f == 0 ? v.x : (f == 1 ? v.y : (f == 2 ? v.z : v.w));
}

// Send tet t's leavers (o[s], per face) to its neighbours: through face f
// into inbox slot src.f of the neighbour (species beyond S written as 0).
template <int SA>
__device__ __forceinline__ void push_inbox(int32_t* __restrict__ in, int4 sr, int S, int Sp, const int4* o) {
    const int slot[4] = {sr.x, sr.y, sr.z, sr.w};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (slot[f] < 0) continue;
        int32_t* d = in + (int64_t)slot[f] * Sp;
        if (SA == 1 || Sp == 1) {
            d[0] = face_of(o[0], f);
        } else if (SA == 2 || Sp == 2) {
            *reinterpret_cast<int2*>(d) = make_int2(face_of(o[0], f), SA > 1 ? face_of(o[SA > 1 ? 1 : 0], f) : 0);
        } else {
#pragma unroll
            for (int q = 0; q < (SA + 3) / 4; ++q) {
                if (4 * q >= Sp) break;
                int v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int s = 4 * q + k;
                    v[k] = (s < S && s < SA) ? face_of(o[s < SA ? s : 0], f) : 0;
                }
                *reinterpret_cast<int4*>(d + 4 * q) = make_int4(v[0], v[1], v[2], v[3]);
            }
        }
    }
}

// Reaction phase of one tet (Algorithm 1, Step 2 and 2.1): Gillespie's
// direct method over [0, tau_k); the first event at or past tau_k is
// discarded.  Before a species' count changes, its occupancy integral
// advances by N * (t_event - t_last).  Under the half-step rule
// (kRuleMid), Nmid receives the counts at tau_k / 2: those after every event
// whose time is below tau_k / 2.  The tet's volume, reaction mask and
// single-precision (N_A V, 1/(N_A V)) come in by value: a non-inlined
// function that took the mesh by reference would pin the caller's copy of
// it in local memory.
static __device__ __noinline__ void react_tet(const ModelParams& mp, int key, uint32_t period, double tau_k,
                                              uint64_t seed, double vol_t, uint32_t on, float2 avf, int64_t* N,
                                              double* occ, double* tl, uint32_t& touched, int64_t* Nmid,
                                              uint32_t* err) {
    const double avv = kAvogadro * (vol_t * 1000.0);
    const bool want_mid = mp.rule == kRuleMid;
    const double half = 0.5 * tau_k;
    bool past_half = false;
    // Per-reaction constants of this tet, computed once: the same values as
    // recomputing them at every event (c = k N_A V, k, or k / (N_A V)).
    double c[kMaxR];
    uint32_t cpos = 0;
    for (int r = 0; r < mp.R; ++r) {
        double kr = mp.k[r];
        int o = mp.order[r];
        c[r] = ((on >> r) & 1u) ? (o == 0 ? kr * avv : (o == 1 ? kr : kr / avv)) : 0.0;
        if (c[r] > 0.0) cpos |= 1u << r;
    }
    rdd::Stream st(seed, (uint32_t)key, period, rdd::kPurposeReaction, 0);
    double tc = 0.0;
    int events = 0;
    for (;;) {
        // propensity a_r = c_r h_r, h_r the number of reactant combinations
        int64_t h[kMaxR];
        bool any = false;
        for (int r = 0; r < mp.R; ++r) {
            int64_t hr = 1;
            int a1 = mp.rs1[r], a2 = mp.rs2[r];
            if (a1 >= 0) {
                if (a2 < 0) hr = N[a1];
                else if (a1 == a2) hr = N[a1] * (N[a1] - 1) / 2;
                else hr = N[a1] * N[a2];
            }
            h[r] = hr;
            any = any || (((cpos >> r) & 1u) && hr != 0);
        }
        if (!any) break;                       // a0 = 0
        const uint64_t x53 = st.bits53();
        // After an event, a single-precision bound often proves that the
        // next event time tc - log(u1)/a0 reaches tau_k (see surely_no_event;
        // here the span is tau_k - tc, kept well above rounding by the
        // 1e-9 guard), which skips the double-precision log and divide.
        if (events > 0) {
            const double span = tau_k - tc;
            if (span > tau_k * 1e-9) {
                float a0f = 0.0f;
                for (int r = 0; r < mp.R; ++r) {
                    if (!((cpos >> r) & 1u) || h[r] == 0) continue;
                    int o = mp.order[r];
                    float cf = o == 0 ? mp.kf[r] * avf.x : (o == 1 ? mp.kf[r] : mp.kf[r] * avf.y);
                    a0f += cf * (float)h[r];
                }
                const uint64_t y = 9007199254740991ull - x53;
                const uint32_t yhi = (uint32_t)(y >> 29);
                const float need = a0f * (float)span * 1.0001f;
                if (yhi != 0u && need < 3.0e38f && (float)yhi * 5.9604644775390625e-08f >= need) break;
            }
        }
        double a[kMaxR];
        double a0 = 0.0;
        for (int r = 0; r < mp.R; ++r) {
            double ar = c[r] * (double)h[r];
            a[r] = ar;
            a0 = a0 + ar;
        }
        const double u1 = ((double)x53 + 1.0) * (1.0 / 9007199254740992.0);
        double tn = tc + (-rdd::own_log(u1)) / a0;
        if (tn >= tau_k) break;
        if (want_mid && !past_half && tn >= half) {
            for (int s = 0; s < mp.S; ++s) Nmid[s] = N[s];
            past_half = true;
        }
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
    if (want_mid && !past_half)
        for (int s = 0; s < mp.S; ++s) Nmid[s] = N[s];
    for (int s = 0; s < mp.S; ++s)
        if ((touched >> s) & 1u) occ[s] = occ[s] + (double)N[s] * (tau_k - tl[s]);
}

// Diffusion of one species out of one tet (Algorithm 1, Step 3; Eq. 2-3;
// Sec. II.B): N* from the occupancy (stochastic rounding of N-bar when the
// count changed during the period, else N), n = min(Binomial(N*, zeta), N),
// split over the faces by conditional binomials; below N* = kMoleculeCut the
// same law one molecule at a time against the cumulative thresholds.  Under
// the half-step comparison rule N* is N(tau_k / 2) (Nmid); under the
// first-order rule the caller passes touched = false, so N* = N(tau_k).
static __device__ __noinline__ int4 diffuse(const double* __restrict__ G, const double* __restrict__ gface, int t,
                                            int key, int s, double Dsp, uint32_t period, double tau_k, uint64_t seed,
                                            int64_t Nt, bool touched, double occ, int64_t Nmid, int32_t rule,
                                            uint4 C) {
    int4 o = make_int4(0, 0, 0, 0);
    double Gt = G[t];
    double z = zeta_of(tau_k, Dsp, Gt);
    if (!(z > 0.0) || Nt <= 0) return o;
    int64_t Nstar = Nt;
    if (touched && rule == kRuleMid) {
        Nstar = Nmid;                          // N(tau_k / 2), an integer: no rounding draw
    } else if (touched) {
        rdd::Stream rs(seed, (uint32_t)key, period, rdd::kPurposeRounding, (uint32_t)s);
        double nbar = occ / tau_k;
        double fl = floor(nbar);
        double frac = nbar - fl;
        Nstar = (int64_t)fl + (rs.u01() < frac ? 1 : 0);
    }
    if (Nstar <= 0) return o;
    rdd::Stream ds(seed, (uint32_t)key, period, rdd::kPurposeDiffusion, (uint32_t)s);
    if (Nstar < kMoleculeCut) {
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
    for (int f = 0; f < 4; ++f) g[f] = gface[4 * t + f];
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

// N[i] for a runtime index without dynamic register indexing (which would
// move the array to local memory).
template <int SA>
__device__ __forceinline__ int32_t pick(const int32_t* N, int i) {
    int32_t v = 0;
#pragma unroll
    for (int k = 0; k < SA; ++k)
        if (k == i) v = N[k];
    return v;
}

// Number of distinct reactant combinations of reaction r as a float (0 when a
// reactant is missing).
template <int SA>
__device__ __forceinline__ float combos_f(const ModelParams& mp, int r, const int32_t* N) {
    int a = mp.rs1[r], b = mp.rs2[r];
    if (a < 0) return 1.0f;
    int32_t na = pick<SA>(N, a);
    if (b < 0) return (float)na;
    if (a == b) return na >= 2 ? 0.5f * (float)na * (float)(na - 1) : 0.0f;
    return (float)na * (float)pick<SA>(N, b);
}

// True only if the exact SSA of this tet would draw no event in this period
// (`on`: the reactions that can fire, in ascending order as the SSA sums
// them):
// with u1 the stream's first uniform, the first event time is
// -log(u1)/a0 >= (1-u1)/a0, so (1-u1) >= a0 tau_k (1 + margin) rules an event
// out.  a0 and the products are evaluated in single precision; their relative
// error (< 3e-6 for 32 reactions) and that of the double-precision path
// (< 1e-13) sit far inside the 1e-4 margin, and 1-u1 is bounded from below by
// truncating its 53-bit integer to 24 bits, so the decision never differs
// from the double-precision one.  Any doubtful case returns false and the
// exact path runs.
template <int SA>
__device__ __forceinline__ bool surely_no_event(const ModelParams& mp, const int32_t* N, uint32_t on, float2 av,
                                                uint32_t period, float tau_kf, uint64_t seed, int key) {
    float a0 = 0.0f;
    for (uint32_t bits = on; bits; bits &= bits - 1u) {
        const int r = __ffs(bits) - 1;
        float h = combos_f<SA>(mp, r, N);
        if (h == 0.0f) continue;
        int o = mp.order[r];
        float c = o == 0 ? mp.kf[r] * av.x : (o == 1 ? mp.kf[r] : mp.kf[r] * av.y);
        a0 += c * h;
    }
    rdd::Stream st(seed, (uint32_t)key, period, rdd::kPurposeReaction, 0);
    uint64_t x = st.bits53();
    uint64_t y = 9007199254740991ull - x;     // (1 - u1) * 2^53
    uint32_t yhi = (uint32_t)(y >> 29);       // top 24 bits: yhi * 2^-24 <= 1 - u1
    if (yhi == 0) return false;
    float lo = (float)yhi * 5.9604644775390625e-08f;
    float need = a0 * tau_kf * 1.0001f;
    return need < 3.0e38f && lo >= need;
}

// One draw per molecule against the cumulative face thresholds (N* < 10 and
// the count untouched by reactions, so N* = N).
__device__ __forceinline__ int4 split_molecules(uint64_t seed, uint32_t period, int key, int sp, int32_t n, uint4 C) {
    int4 o = make_int4(0, 0, 0, 0);
    if (C.w == 0u) return o;                 // nothing can leave (zeta * 2^32 < 1)
    rdd::Stream ds(seed, (uint32_t)key, period, rdd::kPurposeDiffusion, (uint32_t)sp);
    for (int i = 0; i < n; ++i) {
        uint32_t u = ds.u32();
        if (rdd::below(u, C.x)) o.x += 1;
        else if (rdd::below(u, C.y)) o.y += 1;
        else if (rdd::below(u, C.z)) o.z += 1;
        else if (rdd::below(u, C.w)) o.w += 1;
    }
    return o;
}


// The reactions (k > 0, on in the tet, given as `on`) whose reactants are
// present: a species with no molecule rules out every reaction that
// consumes it, one molecule rules out those that consume two.
template <int SA>
__device__ __forceinline__ uint32_t possible_reactions(const ModelParams& mp, const int32_t* N, uint32_t on) {
    uint32_t m = on;
#pragma unroll
    for (int s = 0; s < SA; ++s) {
        if (s >= mp.S) break;
        if (N[s] <= 0) m &= ~mp.needs[s];
        else if (N[s] == 1) m &= ~mp.needs2[s];
    }
    return m;
}

// True when step_tet would run neither non-inlined sampler for this tet:
// every count below kMoleculeCut and, with reactions, no event possible or
// one proved impossible by the single-precision test.  Such a tet gives the
// same result through step_tet<SA, false, false> (nothing touched by
// reactions; only the per-molecule draws).
template <int SA, bool kReact>
__device__ __forceinline__ bool step_is_light(const DevMesh& m, const ModelParams& mp, uint32_t period,
                                              float tau_kf, uint64_t seed, int t, int S, const int32_t* N) {
#pragma unroll
    for (int sp = 0; sp < SA; ++sp) {
        if (sp >= S) break;
        if (N[sp] >= kMoleculeCut) return false;
    }
    if (!kReact) return true;
    const uint32_t on = (mp.has_mask ? m.mask[t] : 0xffffffffu) & mp.kpos;
    const uint32_t poss = possible_reactions<SA>(mp, N, on);
    if (!poss) return true;
    return surely_no_event<SA>(mp, N, poss, m.avv[t], period, tau_kf, seed, key_of(m, t));
}

// Steps 2 and 3 of one period for one tet, given its counts N after the
// previous period's transfers: the reaction phase (skipped when no reaction
// can fire or the single-precision test proves that none fires), then the
// diffusion draws of every species.  On return N holds the molecules that
// stay and o[s] the molecules leaving through each face, except for the
// species whose bit is set in *heavy: those (untouched, 10 <= N < 4096) are
// left for warp_split, which the whole warp must call next.  Returns error
// bits.  With has_pre, `pre` holds species 0's thresholds, already loaded.
// With kCalls = false the non-inlined samplers (react_tet, diffuse) are left
// out: the caller must have checked step_is_light first.
template <int SA, bool kReact, bool kCalls = true>
__device__ __forceinline__ uint32_t step_tet(const DevMesh& m, const ModelParams& mp, uint32_t period, double tau_k,
                                             float tau_kf, uint64_t seed, const uint4* __restrict__ thr, int t,
                                             int S, int32_t* N, int4* o, uint32_t* heavy, uint32_t* err,
                                             int thr_stride = 1, bool has_pre = false,
                                             uint4 pre = make_uint4(0u, 0u, 0u, 0u)) {
    const int64_t T = m.T;
    const int key = key_of(m, t);
    uint32_t bad = 0;
    uint32_t touched = 0;
    double occ[SA];
    int64_t nmid[SA];
    if (kReact && kCalls) {
        uint32_t on = (mp.has_mask ? m.mask[t] : 0xffffffffu) & mp.kpos;
        const uint32_t poss = possible_reactions<SA>(mp, N, on);
        if (poss && !surely_no_event<SA>(mp, N, poss, m.avv[t], period, tau_kf, seed, key)) {
            int64_t N64[SA];
            double tl[SA];
#pragma unroll
            for (int sp = 0; sp < SA; ++sp) {
                if (sp >= S) break;
                N64[sp] = N[sp];
                occ[sp] = 0.0;
                tl[sp] = 0.0;
            }
            react_tet(mp, key, period, tau_k, seed, m.vol[t], mp.has_mask ? m.mask[t] : 0xffffffffu, m.avv[t], N64, occ,
                      tl, touched, nmid, err);
#pragma unroll
            for (int sp = 0; sp < SA; ++sp) {
                if (sp >= S) break;
                int64_t v = N64[sp];
                if (v < 0) { bad |= kErrNegative; v = 0; }
                if (v > 2147483647) { bad |= kErrOverflow; v = 2147483647; }
                N[sp] = (int32_t)v;
            }
        }
    }
#pragma unroll
    for (int sp = 0; sp < SA; ++sp) {
        if (sp >= S) break;
        int32_t Nt = N[sp];
        int4 x = make_int4(0, 0, 0, 0);
        // first-order splitting draws from N(tau_k): the untouched path
        bool tch = kReact && ((touched >> sp) & 1u) && mp.rule != kRuleEnd;
        if (Nt > 0) {
            if (!tch && Nt < kWarpSplitMin) {
                x = split_molecules(seed, period, key, sp, Nt, (has_pre && sp == 0) ? pre : thr[(sp * T + t) * thr_stride]);
            } else if (!tch && Nt < kMoleculeCut) {
                *heavy |= 1u << sp;        // drawn by the whole warp (warp_split)
                o[sp] = x;
                continue;
            } else if (kCalls) {
                x = diffuse(m.G, m.g, t, key, sp, mp.D[sp], period, tau_k, seed, Nt, tch, tch ? occ[sp] : 0.0,
                            tch ? nmid[sp] : (int64_t)Nt, mp.rule,
                            (has_pre && sp == 0) ? pre : thr[(sp * T + t) * thr_stride]);
            }
        }
        o[sp] = x;
        N[sp] = Nt - (x.x + x.y + x.z + x.w);
    }
    return bad;
}


// The per-molecule draw of one (tet, species) spread over a warp: lane l
// computes Philox blocks l, l+32, ... of the tet's diffusion stream (keyed
// by the canonical id `key` of the stored tet t) (block b
// holds the uniforms of molecules 4b..4b+3, exactly the words the sequential
// draw would use) and the face counts are summed over the warp.  Every lane
// of the warp must call this; lanes with heavy == 0 only help.  With has_pre,
// `pre` holds the calling lane's species-0 thresholds, already loaded.
template <int SA>
__device__ __forceinline__ void warp_split(uint32_t heavy, uint64_t seed, uint32_t period, int t, int key,
                                           const uint4* __restrict__ thr, int64_t T, int32_t* N, int4* o,
                                           int thr_stride = 1, bool has_pre = false,
                                           uint4 pre = make_uint4(0u, 0u, 0u, 0u)) {
    const unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned m = __ballot_sync(kAll, heavy != 0u);
        if (m == 0u) break;
        const int src = __ffs(m) - 1;
        const int my_sp = heavy ? __ffs(heavy) - 1 : 0;
        uint4 myC = make_uint4(0, 0, 0, 0);
        if (lane == src) myC = (has_pre && my_sp == 0) ? pre : thr[(my_sp * T + t) * thr_stride];
        const int sp = __shfl_sync(kAll, my_sp, src);
        const int32_t n = __shfl_sync(kAll, pick<SA>(N, my_sp), src);
        const int tt = __shfl_sync(kAll, key, src);
        const uint32_t pr = __shfl_sync(kAll, period, src);
        const uint32_t k0 = __shfl_sync(kAll, (uint32_t)seed, src);
        const uint32_t k1 = __shfl_sync(kAll, (uint32_t)(seed >> 32), src);
        uint4 C;
        C.x = __shfl_sync(kAll, myC.x, src);
        C.y = __shfl_sync(kAll, myC.y, src);
        C.z = __shfl_sync(kAll, myC.z, src);
        C.w = __shfl_sync(kAll, myC.w, src);
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        if (C.w != 0u) {
            const uint32_t tag = (rdd::kPurposeDiffusion << 16) | (uint32_t)sp;
            const int nblocks = (n + 3) >> 2;
            for (int b = lane; b < nblocks; b += 32) {
                uint4 w = rdd::philox_block((uint32_t)b, (uint32_t)tt, pr, tag, k0, k1);
                const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (4 * b + q >= n) break;
                    if (rdd::below(u[q], C.x)) ++c0;
                    else if (rdd::below(u[q], C.y)) ++c1;
                    else if (rdd::below(u[q], C.z)) ++c2;
                    else if (rdd::below(u[q], C.w)) ++c3;
                }
            }
        }
        c0 = __reduce_add_sync(kAll, c0);
        c1 = __reduce_add_sync(kAll, c1);
        c2 = __reduce_add_sync(kAll, c2);
        c3 = __reduce_add_sync(kAll, c3);
        if (lane == src) {
#pragma unroll
            for (int k = 0; k < SA; ++k) {
                if (k == sp) {
                    o[k] = make_int4(c0, c1, c2, c3);
                    N[k] -= c0 + c1 + c2 + c3;
                }
            }
            heavy &= ~(1u << sp);
        }
    }
}


}  // namespace rdk
