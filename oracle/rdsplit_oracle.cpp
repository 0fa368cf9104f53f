// Serial oracle of the operator-split reaction-diffusion method
// (Hepburn, Chen & De Schutter, arXiv:1512.03126, Algorithm 1).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or helper with the CUDA path; it is built with
// -O2 -ffp-contract=off (no FMA contraction, no fast-math) so that every
// floating-point operation is a single IEEE-754 binary64 operation with
// round-to-nearest-even.
//
// Every function below restates one step of the method in the paper's order.
// The readings taken where the paper is silent are listed next to the step.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), one independent stream per
// (seed, period, canonical tet, purpose, species):
//   key     = (seed & 0xffffffff, seed >> 32)
//   counter = (block, tet, period, purpose << 16 | species)
// The words of a stream are consumed in order, four per block.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---------------------------------------------------------------- Philox ----
const uint32_t kPhiloxM0 = 0xD2511F53u;
const uint32_t kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u;   // golden ratio
const uint32_t kPhiloxW1 = 0xBB67AE85u;   // sqrt(3) - 1

// Full product of two words as (high, low) halves.
inline void mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

inline void mulhilo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
    uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    *lo = (p00 & 0xffffffffu) | (mid << 32);
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

// Ten Philox rounds on a 4-word counter, for 32- or 64-bit words (one code
// path, so that pinning the 64-bit member against an independent
// implementation pins the round structure of the 32-bit one).  Each round
// multiplies words 0 and 2 by the two constants, keeps high and low halves,
// and mixes the high halves with words 1 and 3 and the round key; the key is
// bumped by the Weyl constants between rounds.
template <typename W>
void philox_rounds(const W in[4], const W key[2], W M0, W M1, W W0, W W1, W out[4]) {
    W c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3], k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        W h0, l0, h1, l1;
        mulhilo(M0, c0, &h0, &l0);
        mulhilo(M1, c2, &h1, &l1);
        W n0 = h1 ^ c1 ^ k0, n1 = l1, n2 = h0 ^ c3 ^ k1, n3 = l0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void philox4x32_10(const uint32_t in[4], const uint32_t key[2], uint32_t out[4]) {
    philox_rounds<uint32_t>(in, key, kPhiloxM0, kPhiloxM1, kPhiloxW0, kPhiloxW1, out);
}

// The 64-bit-word member of the family (Philox4x64-10).
void philox4x64_10(const uint64_t in[4], const uint64_t key[2], uint64_t out[4]) {
    philox_rounds<uint64_t>(in, key, 0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull, 0x9E3779B97F4A7C15ull,
                            0xBB67AE8584CAA73Bull, out);
}

enum Purpose : uint32_t { kRounding = 0, kDiffusion = 1, kReaction = 2 };

struct Stream {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;

    Stream(uint64_t seed, uint32_t tet, uint32_t period, uint32_t purpose, uint32_t species) {
        key[0] = (uint32_t)(seed & 0xffffffffu);
        key[1] = (uint32_t)(seed >> 32);
        ctr[0] = 0; ctr[1] = tet; ctr[2] = period; ctr[3] = (purpose << 16) | species;
        pos = 4;
    }
    uint32_t u32() {
        if (pos == 4) {
            philox4x32_10(ctr, key, buf);
            ctr[0] += 1;
            pos = 0;
        }
        return buf[pos++];
    }
    // 53-bit integer from two consecutive words: top 27 bits of the first,
    // top 26 bits of the second.
    uint64_t bits53() {
        uint64_t a = u32() >> 5;
        uint64_t b = u32() >> 6;
        return (a << 26) | b;
    }
    // Uniform on [0, 1).
    double u01() { return (double)bits53() * (1.0 / 9007199254740992.0); }
    // Uniform on (0, 1].
    double u01_open0() { return ((double)bits53() + 1.0) * (1.0 / 9007199254740992.0); }
};

// ----------------------------------------------------------- log and exp ----
// Own binary64 log and exp from textbook methods, so that the result path
// uses no libm transcendental.  Only +, -, *, / and exact bit operations.
const double kLn2Hi = 6.93147180369123816490e-01;   // ln 2 with 21 low mantissa bits cleared
const double kLn2Lo = 1.9082149292705877e-10;        // ln 2 - kLn2Hi
const double kInvLn2 = 1.4426950408889634;
const double kSqrt2 = 1.4142135623730951;

uint64_t as_bits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
double from_bits(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }

// log(x), x > 0 finite: x = m 2^e with m in [sqrt(1/2), sqrt(2)); then
// log m = 2 atanh(s), s = (m-1)/(m+1), by its odd power series
// (Abramowitz & Stegun 4.1.27) through s^23; log x = e ln2 + log m with ln2
// split in two parts (Cody & Waite) so that e*kLn2Hi is exact.
double own_log(double x) {
    uint64_t b = as_bits(x);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) {                       // subnormal: scale by 2^54
        x = x * 18014398509481984.0;
        b = as_bits(x);
        e = (int)((b >> 52) & 0x7ff) - 54;
    }
    e -= 1023;
    double m = from_bits((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull);
    if (m > kSqrt2) { m = m * 0.5; e += 1; }
    double f = m - 1.0;
    double s = f / (2.0 + f);
    double z = s * s;
    double p = 1.0 / 23.0;
    for (int j = 10; j >= 0; --j) p = p * z + 1.0 / (double)(2 * j + 1);
    double logm = (s + s) * p;
    double de = (double)e;
    return de * kLn2Hi + (logm + de * kLn2Lo);
}

// exp(x): k = nearest integer to x/ln2, r = x - k ln2 (two-part ln2),
// exp(r) by its Taylor series through r^13 (|r| <= 0.35), times 2^k built
// from the exponent bits.
double own_exp(double x) {
    if (x > 709.0) return std::numeric_limits<double>::infinity();
    if (x < -745.0) return 0.0;
    double kf = std::floor(x * kInvLn2 + 0.5);
    double r = (x - kf * kLn2Hi) - kf * kLn2Lo;
    double fact[14];
    fact[0] = 1.0;
    for (int j = 1; j < 14; ++j) fact[j] = fact[j - 1] * (double)j;
    double p = 1.0 / fact[13];
    for (int j = 12; j >= 0; --j) p = p * r + 1.0 / fact[j];
    int k = (int)kf;
    if (k >= -1022) return p * from_bits((uint64_t)(k + 1023) << 52);
    // result is subnormal: scale in two steps
    return (p * from_bits((uint64_t)(k + 1023 + 64) << 52)) * from_bits((uint64_t)(1023 - 64) << 52);
}

// log(k!) : exact factorial through 18!, Stirling's series with three
// correction terms above (Abramowitz & Stegun 6.1.41).
double log_factorial(int64_t k) {
    if (k < 19) {
        double f = 1.0;
        for (int64_t j = 2; j <= k; ++j) f = f * (double)j;
        return own_log(f);
    }
    double x = (double)k + 1.0;
    double ix = 1.0 / x;
    double ix2 = ix * ix;
    double series = ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0)));
    return (x - 0.5) * own_log(x) - x + 0.91893853320467274 + series;
}

// --------------------------------------------------------------- samplers ---
// Binomial(n, p) by inversion from 0, for n*p < 10 and p <= 1/2: walk the pmf
// f(k+1) = f(k) * (p/q) (n-k)/(k+1) from f(0) = q^n until the uniform is
// used up.  A walk that runs past k = n (only possible through rounding)
// restarts with a new uniform.
int64_t binomial_inversion(int64_t n, double p, Stream& st) {
    double q = 1.0 - p;
    double r = p / q;
    double f0 = own_exp((double)n * own_log(q));
    for (int attempt = 0; attempt < 64; ++attempt) {
        double u = st.u01();
        double f = f0;
        for (int64_t k = 0; k <= n; ++k) {
            if (u < f) return k;
            u = u - f;
            f = f * ((r * (double)(n - k)) / (double)(k + 1));
        }
    }
    return 0;
}

// Binomial(n, p) for n*p >= 10, p <= 1/2: BTRS, the transformed rejection
// with squeeze of W. Hoermann, "The generation of binomial random variates",
// J. Statist. Comput. Simul. 46 (1993).  A candidate k is drawn from the
// hat (a scaled Cauchy-like transform of a uniform); it is accepted at once
// inside the squeeze, else by comparing log(V * hat) with the log of the
// pmf ratio f(k)/f(m) at the mode m.  The loop is bounded (100000 tries,
// then the mode is returned) so that it always terminates.
int64_t binomial_btrs(int64_t n, double p, Stream& st) {
    double q = 1.0 - p;
    double dn = (double)n;
    double spq = std::sqrt(dn * p * q);
    double b = 1.15 + 2.53 * spq;
    double a = -0.0873 + 0.0248 * b + 0.01 * p;
    double c = dn * p + 0.5;
    double vr = 0.92 - 4.2 / b;
    double alpha = (2.83 + 5.1 / b) * spq;
    double lpq = own_log(p / q);
    int64_t m = (int64_t)std::floor((dn + 1.0) * p);
    double h = log_factorial(m) + log_factorial(n - m);
    for (int attempt = 0; attempt < 100000; ++attempt) {
        double u = st.u01() - 0.5;
        double v = st.u01();
        double us = 0.5 - std::fabs(u);
        double kd = std::floor((2.0 * a / us + b) * u + c);
        if (kd < 0.0 || kd > dn) continue;
        int64_t k = (int64_t)kd;
        if (us >= 0.07 && v <= vr) return k;
        double lv = own_log(v * alpha / (a / (us * us) + b));
        double lf = h - log_factorial(k) - log_factorial(n - k) + (double)(k - m) * lpq;
        if (lv <= lf) return k;
    }
    return m;   // unreachable in practice: acceptance probability > 0.5 per try
}

// Binomial(n, p) for any n >= 0, p in [0, 1].
int64_t binomial(int64_t n, double p, Stream& st) {
    if (n <= 0 || p <= 0.0) return 0;
    if (p >= 1.0) return n;
    bool flip = p > 0.5;
    double pp = flip ? 1.0 - p : p;
    int64_t k = ((double)n * pp < 10.0) ? binomial_inversion(n, pp, st) : binomial_btrs(n, pp, st);
    return flip ? n - k : k;
}

// -------------------------------------------------------------- the model ---
const double kAvogadro = 6.02214076e23;
const int64_t kMoleculeCut = 4096;   // one draw per molecule below this N*
const int kMaxSpecies = 16;
const int kMaxReactions = 64;

struct Problem {
    int T, S, R;
    const int32_t* adj;
    const double* vol;
    const double* area;
    const double* dist;
    const double* D;
    const int32_t* lhs;
    const int32_t* rhs;
    const double* k;
    const uint8_t* mask;     // [R][T] or null
    double tau_scale;
    int rule;                // transfer rule: kRuleMean, kRuleEnd or kRuleMid
    int outliers;            // fastest tets left out of the choice of tau (Sec. II.A)
};

// Which count of a period the diffusion draw of Step 3.2 uses (Sec. II.C).
//  kRuleMean  N-bar, the mean occupancy over the period (Eq. 3): the method.
//  kRuleEnd   N(tau_k), the count after the reaction phase: first-order
//             splitting, the comparison method of Sec. III.B (Fig. 7).
//  kRuleMid   N(tau_k / 2), the count at the middle of the period: the
//             "median" reading of N that half-step (Strang) splitting
//             amounts to (Sec. II.C, Fig. 4).
const int kRuleMean = 0;
const int kRuleEnd = 1;
const int kRuleMid = 2;

// Setup (Sec. II.A; Algorithm 1, precompute):
//   g[t][f] = A_tf / (V_t * dist_tf) for faces with a neighbour, else 0;
//   G[t] = g0 + g1 + g2 + g3 (in that order) so that the local diffusion rate
//   of species s is d_st = D_s * G[t] and the face weights are w_f = g_f / G;
//   tau = tau_scale / max over (s, t) of d_st.
// With P.outliers = k > 0 (the outlier option of Sec. II.A: leave the few
// tets with the highest zeta out of the choice of tau), tau = tau_scale /
// d_(k+1), d_(j) the j-th largest of the per-tet rates d_t = max_s d_st; the
// k faster tets then have tau * d_t > 1 and their zeta is capped at 1.
struct Geometry {
    std::vector<double> g, G;
    double tau;
};

Geometry setup_geometry(const Problem& P) {
    Geometry geo;
    geo.g.assign((size_t)P.T * 4, 0.0);
    geo.G.assign(P.T, 0.0);
    std::vector<double> dt(P.T, 0.0);
    for (int t = 0; t < P.T; ++t) {
        double Gt = 0.0;
        for (int f = 0; f < 4; ++f) {
            double gf = 0.0;
            if (P.adj[4 * t + f] >= 0) gf = P.area[4 * t + f] / (P.vol[t] * P.dist[4 * t + f]);
            geo.g[4 * t + f] = gf;
            Gt = Gt + gf;
        }
        geo.G[t] = Gt;
        for (int s = 0; s < P.S; ++s) {
            double d = P.D[s] * Gt;
            if (d > dt[t]) dt[t] = d;
        }
    }
    // the (outliers + 1)-th largest per-tet rate
    std::sort(dt.begin(), dt.end(), [](double a, double b) { return a > b; });
    const double dsel = dt[P.outliers];
    geo.tau = dsel > 0.0 ? P.tau_scale / dsel : std::numeric_limits<double>::infinity();
    return geo;
}

// Transfer probability of one molecule over a period of length tau_k
// (Eq. 1 and the text after it): zeta = tau_k * d, capped at 1.
double zeta_of(double tau_k, double D, double Gt) {
    double z = tau_k * (D * Gt);
    return z > 1.0 ? 1.0 : z;
}

// 32-bit threshold of a cumulative probability y in [0, 1]:
// floor(y 2^32), with 0xffffffff standing for "always" (y >= 1 - 2^-32).
uint32_t threshold_of(double y) {
    double z = y * 4294967296.0;
    if (z >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)z;
}

bool below(uint32_t u, uint32_t C) { return C == 0xffffffffu || u < C; }

// Propensity scale of tet t: N_A * V_t in litres.
double avogadro_volume(double vol_m3) { return kAvogadro * (vol_m3 * 1000.0); }

// Reaction phase of one tet for one period (Algorithm 1, Step 2 and 2.1):
// Gillespie's direct method from 0 to tau_k with the propensities of the
// tet's current counts; an event whose time would reach tau_k is discarded.
// On every event, before the counts change, the occupancy integral of each
// species whose count changes is advanced: occ += N * (t_event - t_last).
// Nmid receives the counts at tau_k / 2: those after every event whose time
// is below tau_k / 2.
void react_tet(const Problem& P, int t, uint32_t period, double tau_k, uint64_t seed,
               int64_t* N, double* occ, double* tlast, bool* touched, int64_t* Nmid) {
    for (int s = 0; s < P.S; ++s) Nmid[s] = N[s];
    if (P.R == 0) return;
    const double half = 0.5 * tau_k;
    bool past_half = false;
    double c[kMaxReactions];
    double avv = avogadro_volume(P.vol[t]);
    for (int r = 0; r < P.R; ++r) {
        int order = 0;
        for (int s = 0; s < P.S; ++s) order += P.lhs[r * P.S + s];
        double kr = P.k[r];
        if (P.mask && P.mask[(size_t)r * P.T + t] == 0) c[r] = 0.0;
        else if (order == 0) c[r] = kr * avv;       // M/s per tet volume -> 1/s
        else if (order == 1) c[r] = kr;             // 1/s
        else c[r] = kr / avv;                       // 1/(M s) -> 1/s per pair
    }
    Stream st(seed, (uint32_t)t, period, kReaction, 0);
    double tc = 0.0;
    for (;;) {
        double a[kMaxReactions];
        double a0 = 0.0;
        for (int r = 0; r < P.R; ++r) {
            // h = number of distinct reactant combinations
            int64_t h = 1;
            for (int s = 0; s < P.S; ++s) {
                int nu = P.lhs[r * P.S + s];
                if (nu == 1) h = h * N[s];
                else if (nu == 2) h = h * (N[s] * (N[s] - 1) / 2);
            }
            a[r] = c[r] * (double)h;
            a0 = a0 + a[r];
        }
        if (!(a0 > 0.0)) break;
        double u1 = st.u01_open0();
        double tn = tc + (-own_log(u1)) / a0;
        if (tn >= tau_k) break;
        if (!past_half && tn >= half) {
            for (int s = 0; s < P.S; ++s) Nmid[s] = N[s];
            past_half = true;
        }
        double target = st.u01() * a0;
        int mu = -1;
        double cum = 0.0;
        for (int r = 0; r < P.R; ++r) {
            cum = cum + a[r];
            if (target < cum) { mu = r; break; }
        }
        if (mu < 0) {
            for (int r = P.R - 1; r >= 0; --r) if (a[r] > 0.0) { mu = r; break; }
        }
        for (int s = 0; s < P.S; ++s) {
            int dn = P.rhs[mu * P.S + s] - P.lhs[mu * P.S + s];
            if (dn != 0) {
                occ[s] = occ[s] + (double)N[s] * (tn - tlast[s]);
                tlast[s] = tn;
                touched[s] = true;
                N[s] += dn;
            }
        }
        tc = tn;
    }
    if (!past_half)
        for (int s = 0; s < P.S; ++s) Nmid[s] = N[s];
    for (int s = 0; s < P.S; ++s)
        if (touched[s]) occ[s] = occ[s] + (double)N[s] * (tau_k - tlast[s]);
}

// Diffusion of one species out of one tet at the end of a period
// (Algorithm 1, Step 3; Eq. 2 and Eq. 3; Sec. II.B).
//  3.1  N-bar = occupancy / tau_k for a species whose count changed during
//       the period; otherwise N-bar = N exactly.  A fractional N-bar is made an
//       integer N* by unbiased stochastic rounding.  Under the comparison
//       rules N* is instead N(tau_k) (kRuleEnd) or N(tau_k / 2) (kRuleMid),
//       both integers, and no rounding draw is made.
//  3.2  n = Binomial(N*, zeta), capped at the molecules present, N(tau_k).
//  3.3  n is split over the faces multinomially by conditional binomials in
//       canonical face order, p_i = w_i / (w_i + ... + w_3), the last face
//       with a neighbour taking the rest.
//  Below N* = kMoleculeCut the same law is drawn one molecule at a time
//  (Sec. II.B, "randomly selecting a direction for each molecule"): each of
//  N* molecules leaves through face f with probability zeta*w_f (as 32-bit
//  thresholds) and stays otherwise; draws stop once N(tau_k) molecules have
//  left.  The paper switches at n = 10 for speed on a CPU; this build
//  switches at 4096, where one draw per molecule spread over a warp is
//  faster on the GPU than the double-precision samplers.
// Step 3.3: n molecules split over the faces multinomially by conditional
// binomials in canonical face order, p_i = g_i / (g_i + ... + g_3), the last
// face with a neighbour taking the rest.
void split_over_faces(const double* g, int64_t n, Stream& st, int64_t out[4]) {
    double suf[4];
    double acc = 0.0;
    for (int f = 3; f >= 0; --f) { acc = g[f] + acc; suf[f] = acc; }
    int last = -1;
    for (int f = 0; f < 4; ++f) if (g[f] > 0.0) last = f;
    int64_t m = n;
    for (int f = 0; f < 4; ++f) {
        if (!(g[f] > 0.0)) continue;
        if (f == last) { out[f] = m; break; }
        int64_t nf = binomial(m, g[f] / suf[f], st);
        out[f] = nf;
        m -= nf;
    }
}

void diffuse_tet_species(const Problem& P, const Geometry& geo, int t, int s, uint32_t period,
                         double tau_k, uint64_t seed, int64_t Nt, bool touched, double occ,
                         int64_t Nmid, int64_t out[4]) {
    out[0] = out[1] = out[2] = out[3] = 0;
    double Gt = geo.G[t];
    double zeta = zeta_of(tau_k, P.D[s], Gt);
    if (!(zeta > 0.0) || Nt <= 0) return;
    int64_t Nstar = Nt;
    if (P.rule == kRuleMid) {
        Nstar = Nmid;
    } else if (P.rule == kRuleMean && touched) {
        Stream rs(seed, (uint32_t)t, period, kRounding, (uint32_t)s);
        double nbar = occ / tau_k;
        double fl = std::floor(nbar);
        double frac = nbar - fl;
        Nstar = (int64_t)fl + (rs.u01() < frac ? 1 : 0);
    }
    if (Nstar <= 0) return;
    const double* g = &geo.g[4 * t];
    Stream st(seed, (uint32_t)t, period, kDiffusion, (uint32_t)s);
    if (Nstar < kMoleculeCut) {
        uint32_t C[4];
        double cum = 0.0;
        for (int f = 0; f < 4; ++f) {
            cum = cum + g[f];
            C[f] = threshold_of(zeta * (cum / Gt));
        }
        int64_t moved = 0;
        for (int64_t i = 0; i < Nstar; ++i) {
            if (moved == Nt) break;
            uint32_t u = st.u32();
            for (int f = 0; f < 4; ++f) {
                if (below(u, C[f])) { out[f] += 1; moved += 1; break; }
            }
        }
        return;
    }
    int64_t n = binomial(Nstar, zeta, st);
    if (n > Nt) n = Nt;
    if (n == 0) return;
    split_over_faces(g, n, st, out);
}

// Validation foils (Sec. II.A, Fig. 2(b, c)): diffusion counts the paper
// shows to lose spatial noise.  Test-only; pure diffusion.
//  kFoilMeanN  n is the discrete mean of the gross transfer, floor(zeta N +
//              1/2), split over the faces multinomially (Fig. 2(b)).
//  kFoilNet    molecules move only with the net flux: through face f to u,
//              the expected gross flows are zeta_t w_tf N_t out and
//              zeta_u w_ur N_u in (r the reverse face); the number sent is
//              binomial with probability max(0, out - in) / N_t per molecule,
//              the faces drawn by conditional binomials (Fig. 2(c), "binomial
//              but based on net diffusive flux").
const int kFoilMeanN = 1;
const int kFoilNet = 2;

void diffuse_foil(const Problem& P, const Geometry& geo, const std::vector<int32_t>& rev,
                  const std::vector<int64_t>& N, int foil, int t, int s, uint32_t period, double tau_k,
                  uint64_t seed, int64_t Nt, int64_t out[4]) {
    out[0] = out[1] = out[2] = out[3] = 0;
    const double Gt = geo.G[t];
    const double zeta = zeta_of(tau_k, P.D[s], Gt);
    if (!(zeta > 0.0) || Nt <= 0) return;
    const double* g = &geo.g[4 * t];
    Stream st(seed, (uint32_t)t, period, kDiffusion, (uint32_t)s);
    if (foil == kFoilMeanN) {
        int64_t n = (int64_t)std::floor(zeta * (double)Nt + 0.5);
        if (n > Nt) n = Nt;
        if (n > 0) split_over_faces(g, n, st, out);
        return;
    }
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f = 0; f < 4; ++f) {
        const int u = P.adj[4 * t + f];
        if (u < 0) continue;
        const double flow_out = zeta * (g[f] / Gt) * (double)Nt;
        const double Gu = geo.G[u];
        const double zu = zeta_of(tau_k, P.D[s], Gu);
        const double flow_in = zu * (geo.g[4 * u + rev[4 * t + f]] / Gu) * (double)N[(size_t)u * P.S + s];
        const double net = flow_out - flow_in;
        p[f] = net > 0.0 ? net / (double)Nt : 0.0;
    }
    int64_t rest = Nt;
    double q = 1.0;
    for (int f = 0; f < 4 && rest > 0; ++f) {
        if (!(p[f] > 0.0)) continue;
        double pf = p[f] / q;
        if (pf > 1.0) pf = 1.0;
        const int64_t x = binomial(rest, pf, st);
        out[f] = x;
        rest -= x;
        q = q - p[f];
        if (!(q > 0.0)) break;
    }
}

// The synchronous transfer (Sec. III.D: changes buffered, then applied):
// N'[t] = rem[t] + sum over faces of what the neighbour sent through the
// shared face.  Returns 0, -2 for a negative count, -3 above 2^31 - 1.
int apply_transfers(int T, int S, const int32_t* adj, const std::vector<int32_t>& rev,
                    const std::vector<int64_t>& rem, const std::vector<int64_t>& out, std::vector<int64_t>& N) {
    for (int t = 0; t < T; ++t)
        for (int s = 0; s < S; ++s) {
            int64_t v = rem[(size_t)t * S + s];
            for (int f = 0; f < 4; ++f) {
                int u = adj[4 * t + f];
                if (u >= 0) v += out[((size_t)u * S + s) * 4 + rev[4 * t + f]];
            }
            if (v < 0) return -2;
            if (v > 2147483647) return -3;
            N[(size_t)t * S + s] = v;
        }
    return 0;
}

}  // namespace

// ------------------------------------------------------------------ C API ---
extern "C" {

void orc_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    philox4x32_10(ctr, key, out);
}
void orc_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
    philox4x64_10(ctr, key, out);
}
void orc_log_many(const double* x, double* y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = own_log(x[i]); }
void orc_exp_many(const double* x, double* y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = own_exp(x[i]); }
void orc_log_factorial_many(const int64_t* k, double* y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = log_factorial(k[i]); }
uint32_t orc_threshold(double y) { return threshold_of(y); }

// Words / uniforms of one stream.
void orc_stream_u32(uint64_t seed, uint32_t tet, uint32_t period, uint32_t purpose, uint32_t species,
                    uint32_t* out, int64_t n) {
    Stream st(seed, tet, period, purpose, species);
    for (int64_t i = 0; i < n; ++i) out[i] = st.u32();
}
void orc_stream_u01(uint64_t seed, uint32_t tet, uint32_t period, uint32_t purpose, uint32_t species,
                    double* out, int64_t n, int open0) {
    Stream st(seed, tet, period, purpose, species);
    for (int64_t i = 0; i < n; ++i) out[i] = open0 ? st.u01_open0() : st.u01();
}

// `count` binomial draws, draw i from its own stream (seed, i, period, purpose, species).
void orc_binomial_many(uint64_t seed, uint32_t period, int64_t n, double p, int64_t* out, int64_t count) {
    for (int64_t i = 0; i < count; ++i) {
        Stream st(seed, (uint32_t)i, period, kDiffusion, 0);
        out[i] = binomial(n, p, st);
    }
}

// tau for a mesh and model (Algorithm 1, precompute).  Returns +inf when no
// species diffuses.
double orc_tau(int32_t T, const int32_t* adj, const double* vol, const double* area,
               const double* dist, int32_t S, const double* D, double tau_scale) {
    Problem P{T, S, 0, adj, vol, area, dist, D, nullptr, nullptr, nullptr, nullptr, tau_scale, kRuleMean, 0};
    return setup_geometry(P).tau;
}

// tau with the `outliers` fastest tets left out of its choice (Sec. II.A);
// NaN for outliers outside [0, T).
double orc_tau_outliers(int32_t T, const int32_t* adj, const double* vol, const double* area,
                        const double* dist, int32_t S, const double* D, double tau_scale, int32_t outliers) {
    if (outliers < 0 || outliers >= T) return std::numeric_limits<double>::quiet_NaN();
    Problem P{T, S, 0, adj, vol, area, dist, D, nullptr, nullptr, nullptr, nullptr, tau_scale, kRuleMean, outliers};
    return setup_geometry(P).tau;
}

// Algorithm 1.  Advances counts [T][S] (in/out) from *t (in/out) towards
// t_end, at most max_periods periods (< 0: no limit).  *period (in/out) is
// the global period index used in the random-number keys.  Returns 0, or a
// negative code: -1 bad arguments, -2 conservation or sign violated,
// -3 int32 overflow.
// `rule` selects the count the diffusion draw uses (kRuleMean, the method;
// kRuleEnd or kRuleMid, the comparison rules of Sec. II.C and III.B).
// `outliers` > 0 takes tau from the (outliers + 1)-th fastest tet (Sec. II.A).
int orc_run_opts(int32_t T, const int32_t* adj, const double* vol, const double* area, const double* dist,
                 int32_t S, const double* D, int32_t R, const int32_t* lhs, const int32_t* rhs,
                 const double* k, const uint8_t* mask, double tau_scale,
                 int32_t* counts, double* t_io, int64_t* period_io, double t_end, uint64_t seed,
                 int64_t max_periods, int32_t rule, int32_t outliers) {
    if (T <= 0 || S <= 0 || S > kMaxSpecies || R < 0 || R > kMaxReactions) return -1;
    if (rule != kRuleMean && rule != kRuleEnd && rule != kRuleMid) return -1;
    if (outliers < 0 || outliers >= T) return -1;
    Problem P{T, S, R, adj, vol, area, dist, D, lhs, rhs, k, mask, tau_scale, rule, outliers};
    Geometry geo = setup_geometry(P);
    std::vector<int64_t> N((size_t)T * S), rem((size_t)T * S), out((size_t)T * S * 4);
    for (size_t i = 0; i < N.size(); ++i) N[i] = counts[i];
    std::vector<int32_t> rev((size_t)T * 4, -1);
    for (int t = 0; t < T; ++t)
        for (int f = 0; f < 4; ++f) {
            int u = adj[4 * t + f];
            if (u < 0) continue;
            for (int r = 0; r < 4; ++r) if (adj[4 * u + r] == t) rev[4 * t + f] = r;
            if (rev[4 * t + f] < 0) return -1;
        }
    std::vector<int64_t> total(S, 0);
    for (int t = 0; t < T; ++t) for (int s = 0; s < S; ++s) total[s] += N[(size_t)t * S + s];
    double t_now = *t_io;
    int64_t period = *period_io;
    int64_t done = 0;
    while (t_now < t_end && (max_periods < 0 || done < max_periods)) {
        // Step 1: align the last period to t_end.
        double tau_k = geo.tau;
        bool last = false;
        if (t_now + geo.tau > t_end) { tau_k = t_end - t_now; last = true; }
        // Step 2 and 3, tet by tet; every draw is keyed by (period, tet), so
        // the order of this loop does not matter.
        for (int t = 0; t < T; ++t) {
            int64_t Nt[kMaxSpecies], Nmid[kMaxSpecies];
            double occ[kMaxSpecies], tl[kMaxSpecies];
            bool touched[kMaxSpecies];
            for (int s = 0; s < S; ++s) {
                Nt[s] = N[(size_t)t * S + s];
                occ[s] = 0.0; tl[s] = 0.0; touched[s] = false;
            }
            react_tet(P, t, (uint32_t)period, tau_k, seed, Nt, occ, tl, touched, Nmid);
            for (int s = 0; s < S; ++s) {
                if (Nt[s] < 0) return -2;
                int64_t o[4];
                diffuse_tet_species(P, geo, t, s, (uint32_t)period, tau_k, seed, Nt[s], touched[s],
                                    occ[s], Nmid[s], o);
                int64_t sum = 0;
                for (int f = 0; f < 4; ++f) { out[((size_t)t * S + s) * 4 + f] = o[f]; sum += o[f]; }
                rem[(size_t)t * S + s] = Nt[s] - sum;
            }
        }
        // Synchronous transfer: every tet keeps what did not leave and
        // receives what its neighbours sent through the shared faces.
        if (int rc = apply_transfers(T, S, adj, rev, rem, out, N)) return rc;
        if (R == 0) {
            for (int s = 0; s < S; ++s) {
                int64_t tot = 0;
                for (int t = 0; t < T; ++t) tot += N[(size_t)t * S + s];
                if (tot != total[s]) return -2;
            }
        }
        // Step 4.
        t_now = last ? t_end : t_now + geo.tau;
        period += 1;
        done += 1;
    }
    for (size_t i = 0; i < N.size(); ++i) counts[i] = (int32_t)N[i];
    *t_io = t_now;
    *period_io = period;
    return 0;
}

// Pure diffusion with a validation foil in place of the binomial count
// (kFoilMeanN or kFoilNet; test-only, Fig. 2).  Same arguments and returns
// as orc_run without reactions.
int orc_run_foil(int32_t T, const int32_t* adj, const double* vol, const double* area, const double* dist,
                 int32_t S, const double* D, double tau_scale, int32_t* counts, double* t_io, int64_t* period_io,
                 double t_end, uint64_t seed, int64_t max_periods, int32_t foil) {
    if (T <= 0 || S <= 0 || S > kMaxSpecies) return -1;
    if (foil != kFoilMeanN && foil != kFoilNet) return -1;
    Problem P{T, S, 0, adj, vol, area, dist, D, nullptr, nullptr, nullptr, nullptr, tau_scale, kRuleMean, 0};
    Geometry geo = setup_geometry(P);
    std::vector<int64_t> N((size_t)T * S), rem((size_t)T * S), out((size_t)T * S * 4);
    for (size_t i = 0; i < N.size(); ++i) N[i] = counts[i];
    std::vector<int32_t> rev((size_t)T * 4, -1);
    for (int t = 0; t < T; ++t)
        for (int f = 0; f < 4; ++f) {
            int u = adj[4 * t + f];
            if (u < 0) continue;
            for (int r = 0; r < 4; ++r) if (adj[4 * u + r] == t) rev[4 * t + f] = r;
            if (rev[4 * t + f] < 0) return -1;
        }
    double t_now = *t_io;
    int64_t period = *period_io;
    int64_t done = 0;
    while (t_now < t_end && (max_periods < 0 || done < max_periods)) {
        double tau_k = geo.tau;
        bool last = false;
        if (t_now + geo.tau > t_end) { tau_k = t_end - t_now; last = true; }
        for (int t = 0; t < T; ++t)
            for (int s = 0; s < S; ++s) {
                int64_t o[4];
                const int64_t Nt = N[(size_t)t * S + s];
                diffuse_foil(P, geo, rev, N, foil, t, s, (uint32_t)period, tau_k, seed, Nt, o);
                int64_t sum = 0;
                for (int f = 0; f < 4; ++f) { out[((size_t)t * S + s) * 4 + f] = o[f]; sum += o[f]; }
                rem[(size_t)t * S + s] = Nt - sum;
            }
        if (int rc = apply_transfers(T, S, adj, rev, rem, out, N)) return rc;
        t_now = last ? t_end : t_now + geo.tau;
        period += 1;
        done += 1;
    }
    for (size_t i = 0; i < N.size(); ++i) counts[i] = (int32_t)N[i];
    *t_io = t_now;
    *period_io = period;
    return 0;
}

// Algorithm 1 with the method's own transfer rule (N-bar, Eq. 3).
int orc_run(int32_t T, const int32_t* adj, const double* vol, const double* area, const double* dist,
            int32_t S, const double* D, int32_t R, const int32_t* lhs, const int32_t* rhs,
            const double* k, const uint8_t* mask, double tau_scale,
            int32_t* counts, double* t_io, int64_t* period_io, double t_end, uint64_t seed,
            int64_t max_periods) {
    return orc_run_opts(T, adj, vol, area, dist, S, D, R, lhs, rhs, k, mask, tau_scale, counts, t_io, period_io,
                        t_end, seed, max_periods, kRuleMean, 0);
}

// Algorithm 1 with a transfer rule and the default choice of tau.
int orc_run_rule(int32_t T, const int32_t* adj, const double* vol, const double* area, const double* dist,
                 int32_t S, const double* D, int32_t R, const int32_t* lhs, const int32_t* rhs,
                 const double* k, const uint8_t* mask, double tau_scale,
                 int32_t* counts, double* t_io, int64_t* period_io, double t_end, uint64_t seed,
                 int64_t max_periods, int32_t rule) {
    return orc_run_opts(T, adj, vol, area, dist, S, D, R, lhs, rhs, k, mask, tau_scale, counts, t_io, period_io,
                        t_end, seed, max_periods, rule, 0);
}

// Steps 2 and 3 of one period (reactions, then the diffusion draws) for the
// tets t_begin .. t_end-1 only, from counts [T][S] (only those tets' rows are
// read).  Writes their out-slots out[(t - t_begin)][S][4] and the molecules
// that stay, rem[(t - t_begin)][S].  This is the per-process work of the
// paper's parallel version (Sec. III.D): each process advances its own part
// of the mesh, then the out-slots on cut faces are exchanged and applied.
int orc_period_tets(int32_t T, const int32_t* adj, const double* vol, const double* area, const double* dist,
                    int32_t S, const double* D, int32_t R, const int32_t* lhs, const int32_t* rhs,
                    const double* k, const uint8_t* mask, double tau_scale, const int32_t* counts,
                    int64_t period, double tau_k, uint64_t seed, int32_t t_begin, int32_t t_end,
                    int32_t* out, int32_t* rem) {
    if (T <= 0 || S <= 0 || S > kMaxSpecies || R < 0 || R > kMaxReactions) return -1;
    if (t_begin < 0 || t_end > T || t_begin > t_end) return -1;
    Problem P{T, S, R, adj, vol, area, dist, D, lhs, rhs, k, mask, tau_scale, kRuleMean, 0};
    Geometry geo = setup_geometry(P);
    for (int t = t_begin; t < t_end; ++t) {
        int64_t Nt[kMaxSpecies], Nmid[kMaxSpecies];
        double occ[kMaxSpecies], tl[kMaxSpecies];
        bool touched[kMaxSpecies];
        for (int s = 0; s < S; ++s) {
            Nt[s] = counts[(size_t)t * S + s];
            occ[s] = 0.0; tl[s] = 0.0; touched[s] = false;
        }
        react_tet(P, t, (uint32_t)period, tau_k, seed, Nt, occ, tl, touched, Nmid);
        for (int s = 0; s < S; ++s) {
            if (Nt[s] < 0) return -2;
            int64_t o[4];
            diffuse_tet_species(P, geo, t, s, (uint32_t)period, tau_k, seed, Nt[s], touched[s], occ[s], Nmid[s], o);
            int64_t sum = 0;
            for (int f = 0; f < 4; ++f) { out[((size_t)(t - t_begin) * S + s) * 4 + f] = (int32_t)o[f]; sum += o[f]; }
            rem[(size_t)(t - t_begin) * S + s] = (int32_t)(Nt[s] - sum);
        }
    }
    return 0;
}

}  // extern "C"
