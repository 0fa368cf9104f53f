// Device-side arithmetic of the operator-splitting period: counter-based
// random streams, binary64 log/exp, and the binomial sampler.
//
// Every function here performs the same sequence of IEEE-754 binary64
// operations as the method's specification (compiled with -fmad=false, so no
// multiply-add contraction), which makes the integer results reproducible
// bit for bit on any conforming implementation of that specification.
#pragma once
#include <stdint.h>

namespace rdd {

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  A stream is keyed by
// the 64-bit seed; its counter is (block, tet, period, purpose<<16|species).
// ------------------------------------------------------------------------
struct Philox {
    static constexpr uint32_t M0 = 0xD2511F53u;
    static constexpr uint32_t M1 = 0xCD9E8D57u;
    static constexpr uint32_t W0 = 0x9E3779B9u;
    static constexpr uint32_t W1 = 0xBB67AE85u;
};

__device__ __forceinline__ uint4 philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0 = __umulhi(Philox::M0, c0), lo0 = Philox::M0 * c0;
        uint32_t hi1 = __umulhi(Philox::M1, c2), lo1 = Philox::M1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += Philox::W0;
        k1 += Philox::W1;
    }
    return make_uint4(c0, c1, c2, c3);
}

enum : uint32_t { kPurposeRounding = 0, kPurposeDiffusion = 1, kPurposeReaction = 2 };

struct Stream {
    uint32_t k0, k1, tet, period, tag;
    uint32_t block;
    uint4 buf;
    int pos;

    __device__ __forceinline__ Stream(uint64_t seed, uint32_t tet_, uint32_t period_, uint32_t purpose,
                                      uint32_t species)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), tet(tet_), period(period_),
          tag((purpose << 16) | species), block(0), pos(4) {}

    __device__ __forceinline__ uint32_t u32() {
        if (pos == 4) {
            buf = philox_block(block, tet, period, tag, k0, k1);
            block += 1;
            pos = 0;
        }
        uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        pos += 1;
        return w;
    }
    __device__ __forceinline__ uint64_t bits53() {
        uint64_t a = u32() >> 5;
        uint64_t b = u32() >> 6;
        return (a << 26) | b;
    }
    // [0, 1)
    __device__ __forceinline__ double u01() { return (double)bits53() * (1.0 / 9007199254740992.0); }
    // (0, 1]
    __device__ __forceinline__ double u01_open0() {
        return ((double)bits53() + 1.0) * (1.0 / 9007199254740992.0);
    }
};

// ------------------------------------------------------------------------
// binary64 log and exp from textbook reductions (only +, -, *, / and exact
// bit operations, so the results do not depend on any math library):
//  log: x = m 2^e, m in [sqrt(1/2), sqrt(2)); log m = 2 atanh((m-1)/(m+1))
//       by its odd power series through degree 23; ln 2 in two parts.
//  exp: x = k ln2 + r (two-part ln 2), exp(r) by Taylor through r^13,
//       scaled by 2^k through the exponent field.
// ------------------------------------------------------------------------
constexpr double kLn2Hi = 6.93147180369123816490e-01;
constexpr double kLn2Lo = 1.9082149292705877e-10;
constexpr double kInvLn2 = 1.4426950408889634;
constexpr double kSqrt2 = 1.4142135623730951;

__device__ __forceinline__ double own_log(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) {
        x = __dmul_rn(x, 18014398509481984.0);
        b = (uint64_t)__double_as_longlong(x);
        e = (int)((b >> 52) & 0x7ff) - 54;
    }
    e -= 1023;
    double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    if (m > kSqrt2) { m = m * 0.5; e += 1; }
    double f = m - 1.0;
    double s = f / (2.0 + f);
    double z = s * s;
    double p = 1.0 / 23.0;
#pragma unroll
    for (int j = 10; j >= 0; --j) p = p * z + 1.0 / (double)(2 * j + 1);
    double logm = (s + s) * p;
    double de = (double)e;
    return de * kLn2Hi + (logm + de * kLn2Lo);
}

__device__ __forceinline__ double own_exp(double x) {
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -745.0) return 0.0;
    double kf = floor(x * kInvLn2 + 0.5);
    double r = (x - kf * kLn2Hi) - kf * kLn2Lo;
    double fact[14];
    fact[0] = 1.0;
#pragma unroll
    for (int j = 1; j < 14; ++j) fact[j] = fact[j - 1] * (double)j;
    double p = 1.0 / fact[13];
#pragma unroll
    for (int j = 12; j >= 0; --j) p = p * r + 1.0 / fact[j];
    int k = (int)kf;
    if (k >= -1022) return p * __longlong_as_double((long long)((uint64_t)(k + 1023) << 52));
    return (p * __longlong_as_double((long long)((uint64_t)(k + 1023 + 64) << 52))) *
           __longlong_as_double((long long)((uint64_t)(1023 - 64) << 52));
}

// log(k!): exact product through 18!, else Stirling's series with three
// correction terms.
__device__ __forceinline__ double log_factorial(int64_t k) {
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

// ------------------------------------------------------------------------
// Binomial(n, p): inversion from 0 when n*min(p,1-p) < 10, otherwise BTRS
// (Hoermann 1993, transformed rejection with squeeze); p > 1/2 is drawn as
// n - Binomial(n, 1-p).
// ------------------------------------------------------------------------
static __device__ __noinline__ int64_t binomial_inversion(int64_t n, double p, Stream& st) {
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

static __device__ __noinline__ int64_t binomial_btrs(int64_t n, double p, Stream& st) {
    double q = 1.0 - p;
    double dn = (double)n;
    double spq = sqrt(dn * p * q);
    double b = 1.15 + 2.53 * spq;
    double a = -0.0873 + 0.0248 * b + 0.01 * p;
    double c = dn * p + 0.5;
    double vr = 0.92 - 4.2 / b;
    double alpha = (2.83 + 5.1 / b) * spq;
    double lpq = own_log(p / q);
    int64_t m = (int64_t)floor((dn + 1.0) * p);
    double h = log_factorial(m) + log_factorial(n - m);
    for (int attempt = 0; attempt < 100000; ++attempt) {
        double u = st.u01() - 0.5;
        double v = st.u01();
        double us = 0.5 - fabs(u);
        double kd = floor((2.0 * a / us + b) * u + c);
        if (kd < 0.0 || kd > dn) continue;
        int64_t k = (int64_t)kd;
        if (us >= 0.07 && v <= vr) return k;
        double lv = own_log(v * alpha / (a / (us * us) + b));
        double lf = h - log_factorial(k) - log_factorial(n - k) + (double)(k - m) * lpq;
        if (lv <= lf) return k;
    }
    return m;
}

__device__ __forceinline__ int64_t binomial(int64_t n, double p, Stream& st) {
    if (n <= 0 || p <= 0.0) return 0;
    if (p >= 1.0) return n;
    bool flip = p > 0.5;
    double pp = flip ? 1.0 - p : p;
    int64_t k = ((double)n * pp < 10.0) ? binomial_inversion(n, pp, st) : binomial_btrs(n, pp, st);
    return flip ? n - k : k;
}

// 32-bit threshold of a cumulative probability; 0xffffffff means "always".
__device__ __forceinline__ uint32_t threshold_of(double y) {
    double z = y * 4294967296.0;
    if (z >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)z;
}

__device__ __forceinline__ bool below(uint32_t u, uint32_t C) { return C == 0xffffffffu || u < C; }

}  // namespace rdd
