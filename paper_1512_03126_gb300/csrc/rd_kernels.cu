// Kernels of the operator-splitting hot path (Algorithm 1 of
// arXiv:1512.03126) for sm_103a.
//
//   k_mesh_setup   face coefficients g = A/(V dist), G = sum g, reverse-face
//                  table, mesh validation, max G           (setup, Sec. II.A)
//   k_tau          tau = tau_scale / max_s(D_s * max_t G_t) (Algorithm 1, precompute)
//   k_thresholds   cumulative 32-bit face thresholds of zeta * w_f
//   k_count_ge     tets with G >= x (rank selection for the outlier option)
//   k_zeta_hist    histogram of zeta over the tets (diagnostic, Fig. 1d)
//   k_period       per tet: gather of the previous period's transfers, SSA
//                  reactions with occupancy (Step 2), mean-corrected binomial
//                  count and multinomial split (Step 3)
//   k_period_light / k_period_slow
//                  the same period in two passes for large meshes: the
//                  common tets without the double-precision samplers, then
//                  the deferred ones with them
//   k_gather       the closing synchronous transfer of a run
//
// Layout: counts and remainders are species-major int32 [S][T] (coalesced);
// transfers go through inboxes int32 [T][4][Sp]: a tet writes what leaves
// through face f into the neighbour's slot (a scattered store that nothing
// waits for) and reads its own four slots, contiguous, in the next period
// (a coalesced load), instead of gathering from its neighbours.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "rd_device.cuh"
#include "rd_internal.h"
#include "rd_period.cuh"

namespace rdk {

namespace {
std::atomic<int64_t> g_launches{0};
constexpr int kBlock = 256;

inline int grid_for(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }
}  // namespace

int64_t launches() { return g_launches.load(); }
void note_launch() { ++g_launches; }

// ---------------------------------------------------------------- setup ----
__global__ void k_mesh_setup(int32_t T, const int32_t* __restrict__ adj, const double* __restrict__ vol,
                             const double* __restrict__ area, const double* __restrict__ dist,
                             int4* __restrict__ src, double* __restrict__ g, double* __restrict__ G,
                             unsigned long long* gmax_bits, uint32_t* err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    uint32_t e = 0;
    double V = vol[t];
    if (!(V > 0.0) || !(V < HUGE_VAL)) e |= kErrVolume;
    int s4[4];
    double gf[4];
    double Gt = 0.0;
    for (int f = 0; f < 4; ++f) {
        int u = adj[4 * t + f];
        s4[f] = -1;
        gf[f] = 0.0;
        if (u >= 0) {
            if (u >= T || u == t) {
                e |= kErrAdjRange;
            } else {
                int slot = -1, hits = 0;
                for (int r = 0; r < 4; ++r)
                    if (adj[4 * u + r] == t) { slot = r; ++hits; }
                if (hits != 1) e |= kErrAdjAsym;
                else s4[f] = 4 * u + slot;
                double A = area[4 * t + f], d = dist[4 * t + f];
                if (!(A >= 0.0) || !(A < HUGE_VAL) || !(d > 0.0) || !(d < HUGE_VAL)) e |= kErrFace;
                else gf[f] = A / (V * d);
            }
        } else if (u != -1) {
            e |= kErrAdjRange;
        }
        Gt = Gt + gf[f];
    }
    src[t] = make_int4(s4[0], s4[1], s4[2], s4[3]);
    for (int f = 0; f < 4; ++f) g[4 * t + f] = gf[f];
    G[t] = Gt;
    if (e) atomicOr(err, e);
    else if (Gt < HUGE_VAL) atomicMax(gmax_bits, (unsigned long long)__double_as_longlong(Gt));
}

void launch_mesh_setup(int32_t T, const int32_t* adj, const double* vol, const double* area,
                       const double* dist, int4* src, double* g, double* G,
                       unsigned long long* gmax_bits, uint32_t* err, cudaStream_t st) {
    k_mesh_setup<<<grid_for(T), kBlock, 0, st>>>(T, adj, vol, area, dist, src, g, G, gmax_bits, err);
    ++g_launches;
}

// Rounding is monotone, so max_{s,t} fl(D_s G_t) = max_s fl(D_s max_t G_t).
__global__ void k_tau(const double* D, int32_t S, const unsigned long long* gmax_bits, double tau_scale,
                      double* tau_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Gmax = __longlong_as_double((long long)*gmax_bits);
    double dmax = 0.0;
    for (int s = 0; s < S; ++s) {
        double d = D[s] * Gmax;
        if (d > dmax) dmax = d;
    }
    *tau_out = dmax > 0.0 ? tau_scale / dmax : __longlong_as_double(0x7ff0000000000000ll);
}

void launch_tau(const double* D, int32_t S, const unsigned long long* gmax_bits, double tau_scale,
                double* tau_out, cudaStream_t st) {
    k_tau<<<1, 32, 0, st>>>(D, S, gmax_bits, tau_scale, tau_out);
    ++g_launches;
}

// Number of tets with G_t >= x (x given by its bit pattern; G >= 0, so bit
// order is value order): one step of the rank selection behind the outlier
// option of Sec. II.A.
__global__ void k_count_ge(int32_t T, const double* __restrict__ G, unsigned long long xbits, unsigned int* count) {
    unsigned int c = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        c += (unsigned long long)__double_as_longlong(G[t]) >= xbits ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

void launch_count_ge(int32_t T, const double* G, unsigned long long xbits, unsigned int* count, cudaStream_t st) {
    k_count_ge<<<std::min(grid_for(T), 1024), kBlock, 0, st>>>(T, G, xbits, count);
    ++g_launches;
}

// Histogram of zeta_t = min(1, tau * (D * G_t)) over the tets (Fig. 1d: the
// fastest species' zeta), bins of width 1/nbins on [0, 1] with zeta = 1 in the
// last; also the sum and the largest value (as bits; zeta >= 0).
__global__ void k_zeta_hist(int32_t T, const double* __restrict__ G, double tau, double D, int32_t nbins,
                            unsigned long long* counts, double* sum, unsigned long long* maxbits) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        double z = tau * (D * G[t]);
        if (z > 1.0) z = 1.0;
        int b = (int)(z * (double)nbins);
        if (b >= nbins) b = nbins - 1;
        atomicAdd(counts + b, 1ull);
        atomicAdd(sum, z);
        atomicMax(maxbits, (unsigned long long)__double_as_longlong(z));
    }
}

void launch_zeta_hist(int32_t T, const double* G, double tau, double D, int32_t nbins, unsigned long long* counts,
                      double* sum, unsigned long long* maxbits, cudaStream_t st) {
    k_zeta_hist<<<std::min(grid_for(T), 1024), kBlock, 0, st>>>(T, G, tau, D, nbins, counts, sum, maxbits);
    ++g_launches;
}

// C_f = floor(2^32 zeta (g_0 + ... + g_f) / G): a molecule leaves through the
// first face f whose threshold exceeds its 32-bit draw, and stays if none does.
__global__ void k_thresholds(int32_t T, ModelParams mp, const double* __restrict__ g,
                             const double* __restrict__ G, double tau_k, uint4* __restrict__ thr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * mp.S) return;
    int s = (int)(i / T);
    int t = (int)(i - (int64_t)s * T);
    double Gt = G[t];
    double z = zeta_of(tau_k, mp.D[s], Gt);
    uint32_t C[4] = {0, 0, 0, 0};
    if (z > 0.0) {
        double cum = 0.0;
        for (int f = 0; f < 4; ++f) {
            cum = cum + g[4 * t + f];
            C[f] = rdd::threshold_of(z * (cum / Gt));
        }
    }
    thr[i] = make_uint4(C[0], C[1], C[2], C[3]);
}

void launch_thresholds(int32_t T, const ModelParams& mp, const double* g, const double* G, double tau_k,
                       uint4* thr, cudaStream_t st) {
    k_thresholds<<<grid_for((int64_t)T * mp.S), kBlock, 0, st>>>(T, mp, g, G, tau_k, thr);
    ++g_launches;
}

__global__ void k_pack_mask(int32_t T, int32_t R, const uint8_t* __restrict__ m8, uint32_t* __restrict__ m32,
                            const int32_t* __restrict__ perm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int c = perm ? perm[t] : t;
    uint32_t bits = 0;
    for (int r = 0; r < R; ++r)
        if (m8[(size_t)r * T + c]) bits |= 1u << r;
    m32[t] = bits;
}

void launch_pack_mask(int32_t T, int32_t R, const uint8_t* mask8, uint32_t* mask32, const int32_t* perm,
                      cudaStream_t st) {
    k_pack_mask<<<grid_for(T), kBlock, 0, st>>>(T, R, mask8, mask32, perm);
    ++g_launches;
}

// Counts between the caller's canonical [T][S] order and the stored [S][T]
// (stored tet t is canonical tet perm[t], or t without a reordering).
__global__ void k_counts_in(int32_t T, int32_t S, const int32_t* __restrict__ ts, int32_t* __restrict__ sm,
                            uint32_t* err, const int32_t* __restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * S) return;
    int t = (int)(i / S), s = (int)(i - (int64_t)t * S);
    const int64_t c = perm ? perm[t] : t;
    int32_t v = ts[c * S + s];
    if (v < 0) { atomicOr(err, kErrNegative); v = 0; }
    sm[(int64_t)s * T + t] = v;
}

__global__ void k_counts_out(int32_t T, int32_t S, const int32_t* __restrict__ sm, int32_t* __restrict__ ts,
                             const int32_t* __restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * S) return;
    int t = (int)(i / S), s = (int)(i - (int64_t)t * S);
    const int64_t c = perm ? perm[t] : t;
    ts[c * S + s] = sm[(int64_t)s * T + t];
}

void launch_counts_in(int32_t T, int32_t S, const int32_t* ts, int32_t* sm, uint32_t* err, const int32_t* perm,
                      cudaStream_t st) {
    k_counts_in<<<grid_for((int64_t)T * S), kBlock, 0, st>>>(T, S, ts, sm, err, perm);
    ++g_launches;
}

void launch_counts_out(int32_t T, int32_t S, const int32_t* sm, int32_t* ts, const int32_t* perm, cudaStream_t st) {
    k_counts_out<<<grid_for((int64_t)T * S), kBlock, 0, st>>>(T, S, sm, ts, perm);
    ++g_launches;
}

// ---------------------------------------------------------------- period ---
void finish_model_params(ModelParams& mp) {
    mp.kpos = 0;
    for (int s = 0; s < kMaxS; ++s) mp.needs[s] = mp.needs2[s] = 0u;
    for (int r = 0; r < mp.R; ++r) {
        mp.rs1[r] = mp.rs2[r] = -1;
        for (int s = 0; s < mp.S; ++s) {
            if (mp.lhs[r][s] == 2) { mp.rs1[r] = mp.rs2[r] = (int8_t)s; }
            else if (mp.lhs[r][s] == 1) {
                if (mp.rs1[r] < 0) mp.rs1[r] = (int8_t)s;
                else mp.rs2[r] = (int8_t)s;
            }
        }
        mp.kf[r] = (float)mp.k[r];
        if (mp.k[r] > 0.0) mp.kpos |= 1u << r;
        for (int s = 0; s < mp.S; ++s) {
            if (mp.lhs[r][s] >= 1) mp.needs[s] |= 1u << r;
            if (mp.lhs[r][s] >= 2) mp.needs2[s] |= 1u << r;
        }
    }
}

__global__ void k_avv(int32_t T, const double* __restrict__ vol, float2* __restrict__ avv) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double a = kAvogadro * (vol[t] * 1000.0);
    avv[t] = make_float2((float)a, (float)(1.0 / a));
}

void launch_avv(int32_t T, const double* vol, float2* avv, cudaStream_t st) {
    k_avv<<<grid_for(T), kBlock, 0, st>>>(T, vol, avv);
    ++g_launches;
}

// A tet's counts at the start of a period: its molecules that stayed in the
// previous period plus what its neighbours sent (its inbox), or the counts
// of the handle in a run's first period.  Returns error bits.
template <int SA>
__device__ __forceinline__ uint32_t gather_counts(const DevState& s, const PeriodArgs& a, int t, int T, int S, int Sp,
                                                  int32_t* N) {
    uint32_t bad = 0;
    int64_t n[SA];
#pragma unroll
    for (int sp = 0; sp < SA; ++sp) {
        if (sp >= S) break;
        n[sp] = a.first ? s.cnt[(int64_t)sp * T + t] : s.rem[(int64_t)sp * T + t];
    }
    if (!a.first) add_inbox<SA>(a.in_prev, t, S, Sp, n);
#pragma unroll
    for (int sp = 0; sp < SA; ++sp) {
        if (sp >= S) break;
        int64_t v = n[sp];
        if (v > 2147483647) { bad |= kErrOverflow; v = 2147483647; }
        if (v < 0) { bad |= kErrNegative; v = 0; }
        N[sp] = (int32_t)v;
    }
    return bad;
}

// One period for one tet: apply the previous period's transfers, run the
// reaction phase, draw the diffusion out-counts.  S_ > 0 fixes the species
// count at compile time so that counts live in registers; S_ = 0 reads it
// from the model (up to kMaxS).
template <int S_, bool kReact>
__global__ void __launch_bounds__(kBlock) k_period(DevMesh m, ModelParams mp, DevState s, PeriodArgs a) {
    constexpr int SA = S_ > 0 ? S_ : kMaxS;
    const int S = S_ > 0 ? S_ : mp.S;
    const int t_hi = a.t_hi > 0 ? a.t_hi : m.T;
    const int t = a.t_lo + blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < t_hi;         // every lane stays for the warp draw
    const int T = m.T;
    const int Sp = inbox_stride(S);
    int32_t N[SA];
    int4 o[SA];
    int4 sr = make_int4(-1, -1, -1, -1);
    uint32_t bad = 0, heavy = 0;
    if (valid) {
        sr = m.src[t];
        bad |= gather_counts<SA>(s, a, t, T, S, Sp, N);
        bad |= step_tet<SA, kReact>(m, mp, a.period, a.tau_k, a.tau_kf, a.seed, a.thr, t, S, N, o, &heavy, s.err);
    }
    warp_split<SA>(heavy, a.seed, a.period, t, valid ? key_of(m, t) : 0, a.thr, T, N, o);
    if (valid) {
        push_inbox<SA>(a.in_cur, sr, S, Sp, o);
#pragma unroll
        for (int sp = 0; sp < SA; ++sp) {
            if (sp >= S) break;
            s.rem[(int64_t)sp * T + t] = N[sp];
        }
        if (bad) atomicOr(s.err, bad);
    }
}

template <int S_>
void launch_period_s(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a, int block,
                     cudaStream_t st) {
    const int64_t n = (a.t_hi > 0 ? a.t_hi : m.T) - a.t_lo;
    const int grid = (int)((n + block - 1) / block);
    if (mp.any_reaction) k_period<S_, true><<<grid, block, 0, st>>>(m, mp, s, a);
    else k_period<S_, false><<<grid, block, 0, st>>>(m, mp, s, a);
}

void launch_period(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a, int block,
                   cudaStream_t st) {
    switch (mp.S) {
        case 1: launch_period_s<1>(m, mp, s, a, block, st); break;
        case 2: launch_period_s<2>(m, mp, s, a, block, st); break;
        case 3: launch_period_s<3>(m, mp, s, a, block, st); break;
        case 4: launch_period_s<4>(m, mp, s, a, block, st); break;
        case 8: launch_period_s<8>(m, mp, s, a, block, st); break;
        default: launch_period_s<0>(m, mp, s, a, block, st); break;
    }
    ++g_launches;
}

// The same period split in two passes, for large meshes.  The light pass
// runs every tet that needs neither the reaction phase (no reaction
// possible, or one proved impossible by the single-precision test) nor the
// double-precision binomial (all counts below kMoleculeCut): it is compiled
// without the non-inlined samplers, so it holds fewer registers and more
// warps per SM.  It defers every other tet to a queue, with its gathered
// counts stored in rem; the slow pass runs the queued tets with the full
// step.  Every draw is keyed by (tet, period), so the result equals the
// fused kernel's.  queue holds T entries; qcount[parity] counts this
// period's, and the light pass clears the other parity's for the next.
template <int S_, bool kReact>
__global__ void __launch_bounds__(kBlock, 3) k_period_light(DevMesh m, ModelParams mp, DevState s, PeriodArgs a,
                                                            int32_t* __restrict__ queue, int32_t* qcount,
                                                            int32_t parity) {
    constexpr int SA = S_ > 0 ? S_ : kMaxS;
    const int S = S_ > 0 ? S_ : mp.S;
    const int t_hi = a.t_hi > 0 ? a.t_hi : m.T;
    const int t = a.t_lo + blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < t_hi;         // every lane stays for the warp draw
    const int T = m.T;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) qcount[parity ^ 1] = 0;
    const int Sp = inbox_stride(S);
    int32_t N[SA];
    int4 o[SA];
    int4 sr = make_int4(-1, -1, -1, -1);
    uint32_t bad = 0, heavy = 0;
    bool light = false;
    if (valid) {
        sr = m.src[t];
        bad |= gather_counts<SA>(s, a, t, T, S, Sp, N);
        light = step_is_light<SA, kReact>(m, mp, a.period, a.tau_kf, a.seed, t, S, N);
        if (light) {
            bad |= step_tet<SA, false, false>(m, mp, a.period, a.tau_k, a.tau_kf, a.seed, a.thr, t, S, N, o, &heavy,
                                              s.err);
        } else {
#pragma unroll
            for (int sp = 0; sp < SA; ++sp) {
                if (sp >= S) break;
                s.rem[(int64_t)sp * T + t] = N[sp];
            }
        }
    }
    // deferred tets: one queue slot reservation per warp
    const unsigned dm = __ballot_sync(0xffffffffu, valid && !light);
    if (dm) {
        const int leader = __ffs(dm) - 1;
        int at = 0;
        if (lane == leader) at = atomicAdd(qcount + parity, __popc(dm));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (valid && !light) queue[at + __popc(dm & ((1u << lane) - 1u))] = t;
    }
    warp_split<SA>(heavy, a.seed, a.period, t, valid ? key_of(m, t) : 0, a.thr, T, N, o);
    if (valid && light) {
        push_inbox<SA>(a.in_cur, sr, S, Sp, o);
#pragma unroll
        for (int sp = 0; sp < SA; ++sp) {
            if (sp >= S) break;
            s.rem[(int64_t)sp * T + t] = N[sp];
        }
    }
    if (bad) atomicOr(s.err, bad);
}

// The queued tets of one period with the full step (reaction phase and the
// double-precision samplers), warp by warp over the queue.
template <int S_, bool kReact>
__global__ void __launch_bounds__(kBlock) k_period_slow(DevMesh m, ModelParams mp, DevState s, PeriodArgs a,
                                                        const int32_t* __restrict__ queue, const int32_t* qcount,
                                                        int32_t parity) {
    constexpr int SA = S_ > 0 ? S_ : kMaxS;
    const int S = S_ > 0 ? S_ : mp.S;
    const int T = m.T;
    const int n = qcount[parity];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < n; base += nw * 32) {
        const bool live = base + lane < n;
        const int t = live ? queue[base + lane] : 0;
        int32_t N[SA];
        int4 o[SA];
        uint32_t bad = 0, heavy = 0;
        if (live) {
#pragma unroll
            for (int sp = 0; sp < SA; ++sp) {
                if (sp >= S) break;
                N[sp] = s.rem[(int64_t)sp * T + t];
            }
            bad |= step_tet<SA, kReact>(m, mp, a.period, a.tau_k, a.tau_kf, a.seed, a.thr, t, S, N, o, &heavy, s.err);
        }
        warp_split<SA>(heavy, a.seed, a.period, t, live ? key_of(m, t) : 0, a.thr, T, N, o);
        if (live) {
            push_inbox<SA>(a.in_cur, m.src[t], S, inbox_stride(S), o);
#pragma unroll
            for (int sp = 0; sp < SA; ++sp) {
                if (sp >= S) break;
                s.rem[(int64_t)sp * T + t] = N[sp];
            }
        }
        if (bad) atomicOr(s.err, bad);
    }
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <int S_>
void launch_split_s(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a,
                    int32_t* queue, int32_t* qcount, int32_t parity, int block, cudaStream_t st) {
    const int64_t n = (a.t_hi > 0 ? a.t_hi : m.T) - a.t_lo;
    const int grid = (int)((n + block - 1) / block);
    const int grid_slow = std::min(grid_for(m.T), 2 * sm_count());
    if (mp.any_reaction) {
        k_period_light<S_, true><<<grid, block, 0, st>>>(m, mp, s, a, queue, qcount, parity);
        k_period_slow<S_, true><<<grid_slow, kBlock, 0, st>>>(m, mp, s, a, queue, qcount, parity);
    } else {
        k_period_light<S_, false><<<grid, block, 0, st>>>(m, mp, s, a, queue, qcount, parity);
        k_period_slow<S_, false><<<grid_slow, kBlock, 0, st>>>(m, mp, s, a, queue, qcount, parity);
    }
}

void launch_period_split(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a,
                         int32_t* queue, int32_t* qcount, int32_t parity, int block, cudaStream_t st) {
    switch (mp.S) {
        case 1: launch_split_s<1>(m, mp, s, a, queue, qcount, parity, block, st); break;
        case 2: launch_split_s<2>(m, mp, s, a, queue, qcount, parity, block, st); break;
        case 3: launch_split_s<3>(m, mp, s, a, queue, qcount, parity, block, st); break;
        case 4: launch_split_s<4>(m, mp, s, a, queue, qcount, parity, block, st); break;
        case 8: launch_split_s<8>(m, mp, s, a, queue, qcount, parity, block, st); break;
        default: launch_split_s<0>(m, mp, s, a, queue, qcount, parity, block, st); break;
    }
    g_launches += 2;
}

__global__ void k_gather(DevMesh m, int32_t S, DevState s, const int32_t* __restrict__ in_last, int32_t t_lo,
                         int32_t t_hi) {
    int t = t_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= t_hi) return;
    const int T = m.T;
    const int Sp = inbox_stride(S);
    const int32_t* box = in_last + (int64_t)t * 4 * Sp;
    uint32_t bad = 0;
    for (int sp = 0; sp < S; ++sp) {
        int64_t n = s.rem[(int64_t)sp * T + t];
        for (int f = 0; f < 4; ++f) n += box[f * Sp + sp];
        if (n > 2147483647) { bad |= kErrOverflow; n = 2147483647; }
        if (n < 0) { bad |= kErrNegative; n = 0; }
        s.cnt[(int64_t)sp * T + t] = (int32_t)n;
    }
    if (bad) atomicOr(s.err, bad);
}

void launch_gather(const DevMesh& m, int32_t S, const DevState& s, const int32_t* in_last, cudaStream_t st,
                   int32_t t_lo, int32_t t_hi) {
    if (t_hi <= 0) t_hi = m.T;
    k_gather<<<grid_for(t_hi - t_lo), kBlock, 0, st>>>(m, S, s, in_last, t_lo, t_hi);
    ++g_launches;
}

__global__ void k_inbox_export(int32_t S, const int32_t* __restrict__ inbox, const int32_t* __restrict__ slots,
                               int32_t n, int32_t* __restrict__ buf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * S) return;
    const int64_t k = i / S, sp = i - k * S;
    buf[i] = inbox[(int64_t)slots[k] * inbox_stride(S) + sp];
}

__global__ void k_inbox_import(int32_t S, int32_t* __restrict__ inbox, const int32_t* __restrict__ slots,
                               int32_t n, const int32_t* __restrict__ buf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * S) return;
    const int64_t k = i / S, sp = i - k * S;
    inbox[(int64_t)slots[k] * inbox_stride(S) + sp] = buf[i];
}

void launch_inbox_export(int32_t S, const int32_t* inbox, const int32_t* slots, int32_t n, int32_t* buf,
                         cudaStream_t st) {
    if (n <= 0) return;
    k_inbox_export<<<grid_for((int64_t)n * S), kBlock, 0, st>>>(S, inbox, slots, n, buf);
    ++g_launches;
}

void launch_inbox_import(int32_t S, int32_t* inbox, const int32_t* slots, int32_t n, const int32_t* buf,
                         cudaStream_t st) {
    if (n <= 0) return;
    k_inbox_import<<<grid_for((int64_t)n * S), kBlock, 0, st>>>(S, inbox, slots, n, buf);
    ++g_launches;
}

}  // namespace rdk
