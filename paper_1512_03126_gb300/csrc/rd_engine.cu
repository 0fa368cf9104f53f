// Batched engine: many independent simulations (mesh handles) advanced by one
// persistent kernel, touching only tets that hold molecules.
//
// Realisations run in parallel are the embarrassingly parallel use of the
// method (Sec. I of arXiv:1512.03126).  Each thread-block cluster takes one
// simulation from a work queue (largest first) and runs its periods of
// Algorithm 1 itself, with cluster.sync() as the period barrier, so that no
// grid-wide synchronisation and no spin-wait is needed.  Per period the
// cluster visits the tets whose bit is set in that period's activity bitmap
// (tets that hold molecules or have a zero-order reaction on), runs the same
// per-tet work as the dense kernel (step_tet, warp_split), and adds the
// molecules that stay or leave into the next count buffer with integer atomic
// adds — exact and independent of order, so the counts equal those of the
// dense gather.  A tet that keeps or receives molecules sets its bit in the
// next period's bitmap.  One simulation's active region is touched by one
// cluster only, which keeps it in those SMs' L1 and in L2.
//
// The random streams of a simulation are keyed by its own seed, period index
// and canonical tet ids, so its counts do not depend on what runs beside it.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <vector>

#include "rd_api_internal.h"
#include "rd_device.cuh"
#include "rd_internal.h"
#include "rd_period.cuh"

using namespace rdk;

namespace {

constexpr int kRunBlock = 512;

struct SlotDesc {
    DevMesh m;
    const uint4* thr;        // thresholds for tau
    const uint4* thr_last;   // thresholds for the shortened last period
    int32_t* N[2];           // count buffers [S][T]; the slice starts in N[0]
    uint32_t* bits[2];       // active-tet bitmaps (bit t of word t/32), by period parity in the slice
    const uint4* packed;     // one species: {src, thr} per tet (null: separate arrays)
    int32_t* N2;             // one species: counts of both parities interleaved (null: N[2])
    uint64_t seed;
    uint32_t period0;        // global period index of local period 0
    int32_t P;               // periods to run in total
    int32_t q0, q1;          // this slice runs local periods q0 .. q1-1
    int32_t last_short;      // local period P-1 is shortened
    int32_t S;
    uint32_t zero_order;     // reactions of order 0 with k > 0
    double tau, tau_last;
    float tauf, tau_lastf;
};

__device__ __forceinline__ bool zero_order_on(const SlotDesc& d, const ModelParams& mp, int t) {
    if (!d.zero_order) return false;
    uint32_t on = mp.has_mask ? d.m.mask[t] : 0xffffffffu;
    return (on & d.zero_order) != 0u;
}

// Fire-and-forget integer add to global memory (no value comes back, so the
// warp does not wait for the L2 round trip).
__device__ __forceinline__ void red_add(int32_t* p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v));
}

// Device clock in nanoseconds (the global timer shared by all SMs).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Fire-and-forget OR into a global bitmap word.
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v));
}

constexpr int kWarps = kRunBlock / 32;
constexpr int kGroup = 8;                   // bitmap columns (32 words each) a warp loads at once
constexpr int kQueue = 64;                  // deferred tets per warp
constexpr int kListCap = 32 * 32 + 32;      // active tets one column can add, plus a partial round
constexpr int kDynSmemBytes = kWarps * kListCap * 4;

// Shared memory of the engine kernel, at file scope so that the period
// functions below address it directly.
__shared__ int32_t s_item;                          // work-item index (first CTA of the cluster)
__shared__ unsigned long long s_mass[3];            // [0] molecules of the simulation (all species) at the
                                                    // start of the period; [1], [2] net change by reactions
                                                    // in periods of even / odd parity (two's complement)
__shared__ uint32_t s_wbuf[kWarps][kGroup * 32];    // per warp: the bitmap words of its current batch
__shared__ int32_t s_slowq[kWarps][kQueue];         // per warp: tets deferred to the rounds with the full step
extern __shared__ int32_t s_list[];                 // [kWarps][kListCap]: per warp, active tets not yet run

// Where one period stands for one warp.  The light pass stops early when the
// warp's queue of deferred tets could overflow, and resumes after the queue
// has been run: at batch g0, column kk (the batch's words are kept in s_wbuf
// when `loaded`), with `cnt` active tets still in the warp's list.
struct LightState {
    uint32_t bad;
    int32_t n_slow;      // tets in the warp's queue
    int32_t g0, kk;      // resume point (batch, column)
    int32_t cnt;         // tets in the warp's list
    int32_t loaded;      // the batch's words are in s_wbuf
    int32_t finished;
    unsigned long long done;
};

// Everything a period pass derives from the slot descriptor and the period.
template <int kC>
struct PeriodView {
    int T, S, W, r, tstride;
    bool use_packed, more;
    double tau_k;
    float tau_kf;
    uint32_t period;
    const uint4* thr;
    int32_t* Ncur;
    int32_t* Nnext;
    uint32_t* bcur;
    uint32_t* bnext;
    int64_t cstride;

    __device__ __forceinline__ PeriodView(const SlotDesc& d, int q) {
        T = d.m.T;
        S = d.S;
        W = (T + 31) >> 5;
        r = (q - d.q0) & 1;
        const bool last = (q == d.P - 1) && d.last_short;
        tau_k = last ? d.tau_last : d.tau;
        tau_kf = last ? d.tau_lastf : d.tauf;
        // thresholds: packed beside the reverse-face record (stride 2) except
        // in a shortened last period
        use_packed = d.packed != nullptr && !last;
        thr = last ? d.thr_last : (use_packed ? d.packed + 1 : d.thr);
        tstride = use_packed ? 2 : 1;
        period = d.period0 + (uint32_t)q;
        // counts of this period and the next: N[r] / N[r^1], or the two
        // halves of the interleaved pairs
        const bool inter = d.N2 != nullptr;
        Ncur = inter ? d.N2 + r : d.N[r];
        Nnext = inter ? d.N2 + (r ^ 1) : d.N[r ^ 1];
        cstride = inter ? 2 : 1;
        bcur = d.bits[r];
        bnext = d.bits[r ^ 1];
        more = q + 1 < d.q1;
    }

    // Transfer of one tet's molecules (kept and leaving) into the next
    // counts (fire-and-forget integer adds), and its bits in the next bitmap
    // (fire-and-forget ORs: a bit set twice is set once).  An add that takes
    // a count past 2^31-1 wraps it negative; as the simulation's molecule
    // total is kept below 2^32 (checked every period), the next read of the
    // count, or the check at the end of the slice, sees it negative and
    // reports the overflow, exactly when the dense gather would.
    template <int SA, bool kReact>
    __device__ __forceinline__ uint32_t scatter(const SlotDesc& d, const ModelParams& mp, int t, const int4& sr,
                                                const int32_t* N, const int4* o) const {
        uint32_t bad = 0;
        const int nbr[4] = {sr.x, sr.y, sr.z, sr.w};
        bool keep = kReact && zero_order_on(d, mp, t);
        bool send[4] = {false, false, false, false};
#pragma unroll
        for (int s = 0; s < SA; ++s) {
            if (s >= S) break;
            int32_t* Ns = Nnext + (int64_t)s * T * cstride;
            if (N[s] > 0) {
                red_add(Ns + (int64_t)t * cstride, N[s]);
                keep = true;
            }
            const int ov[4] = {o[s].x, o[s].y, o[s].z, o[s].w};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (ov[f] <= 0) continue;
                if (nbr[f] < 0) { bad |= kErrNegative; continue; }
                red_add(Ns + (int64_t)(nbr[f] >> 2) * cstride, ov[f]);
                send[f] = true;
            }
        }
        if (more) {
            if (keep) red_or(bnext + (t >> 5), 1u << (t & 31));
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!send[f]) continue;
                const int u = nbr[f] >> 2;
                red_or(bnext + (u >> 5), 1u << (u & 31));
            }
        }
        return bad;
    }
};

// The light pass of one period for one warp.  The bitmap is dealt to the
// cluster's kW warps in runs of 4 words (128 tets): run r goes to warp
// r mod kW, so the active tets of a region are spread over all warps (runs
// of 4 measured faster than runs of 1, 2 or 8).  A column is 8 runs of a
// warp (32 words, one per lane); a warp
// loads kGroup of its columns at once, clears them for their next use, and
// appends the set bits of each column to its list in shared memory
// (a prefix sum of the lanes' popcounts gives each lane its place); whenever
// the list holds 32 tets, one round takes them, one per lane.  A round runs
// every tet that needs neither a non-inlined sampler (step_is_light) nor a
// whole-warp draw (10 or more molecules of a species) with the call-free
// step, and queues the others for the slow pass.  Kept out of
// line, and free of calls, so that the compiler allocates its registers
// without the double-precision samplers' demands.  Returns early, with a
// resume point, when the next round could overflow the queue.
template <int SA, bool kReact, int kC>
__device__ __noinline__ LightState light_pass(const SlotDesc* __restrict__ dp, const ModelParams* __restrict__ mpp,
                                              int q, uint32_t* err, LightState st) {
    constexpr unsigned kAll = 0xffffffffu;
    constexpr int kW = kC * kWarps;
    const SlotDesc& d = *dp;
    const ModelParams& mp = *mpp;
    const PeriodView<kC> v(d, q);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rank = kC > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    const int gw = rank * kWarps + warp;
    const unsigned lane_lt = (1u << lane) - 1u;
    uint32_t* wb = s_wbuf[warp];
    int32_t* list = s_list + warp * kListCap;
    int32_t* slowq = s_slowq[warp];
    st.bad = 0u;
    st.n_slow = 0;
    st.done = 0ull;

    // one round: the tets t of the live lanes
    auto round = [&](int t, bool live) {
        uint32_t heavy = 0;
        int32_t N[SA];
        int4 o[SA];
        int4 sr = make_int4(-1, -1, -1, -1);
        uint4 pre = make_uint4(0u, 0u, 0u, 0u);
        bool light = false;
        if (live) {
            // the tet's record and counts, loaded together
            sr = d.packed ? *reinterpret_cast<const int4*>(d.packed + 2 * t) : d.m.src[t];
            if (v.use_packed) pre = d.packed[2 * t + 1];
#pragma unroll
            for (int s = 0; s < SA; ++s) {
                if (s >= v.S) break;
                N[s] = v.Ncur[((int64_t)s * v.T + t) * v.cstride];
                if (N[s] < 0) {          // wrapped past 2^31-1 by the previous period's adds
                    st.bad |= kErrOverflow;
                    N[s] = 0;
                }
            }
            light = step_is_light<SA, kReact>(d.m, mp, v.period, v.tau_kf, d.seed, t, v.S, N);
            // tets whose draws need the whole warp (warp_split) go to the slow
            // pass too, which keeps the light pass free of that loop
#pragma unroll
            for (int s = 0; s < SA; ++s) {
                if (s >= v.S) break;
                if (N[s] >= kWarpSplitMin) light = false;
            }
        }
        const unsigned slow_mask = __ballot_sync(kAll, live && !light);
        if (live && !light) slowq[st.n_slow + __popc(slow_mask & lane_lt)] = t;
        st.n_slow += __popc(slow_mask);
        if (light) {
#pragma unroll
            for (int s = 0; s < SA; ++s) {
                if (s >= v.S) break;
                v.Ncur[((int64_t)s * v.T + t) * v.cstride] = 0;
            }
            if (SA == 1 && !kReact && v.use_packed && N[0] <= 4) {
                // one species, at most four molecules: the first Philox
                // block of the tet's diffusion stream holds all their draws
                // (the words split_molecules would take, in its order)
                const uint32_t key = (uint32_t)key_of(d.m, t);
                const uint4 w = rdd::philox_block(0u, key, v.period, rdd::kPurposeDiffusion << 16,
                                                  (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
                const uint32_t u[4] = {w.x, w.y, w.z, w.w};
                int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= N[0]) break;
                    if (rdd::below(u[i], pre.x)) ++c0;
                    else if (rdd::below(u[i], pre.y)) ++c1;
                    else if (rdd::below(u[i], pre.z)) ++c2;
                    else if (rdd::below(u[i], pre.w)) ++c3;
                }
                o[0] = make_int4(c0, c1, c2, c3);
                N[0] -= c0 + c1 + c2 + c3;
            } else {
                st.bad |= step_tet<SA, false, false>(d.m, mp, v.period, v.tau_k, v.tau_kf, d.seed, v.thr, t, v.S, N,
                                                     o, &heavy, err, v.tstride, v.use_packed, pre);
            }
        }
        if (light) st.bad |= v.template scatter<SA, kReact>(d, mp, t, sr, N, o);
    };

    // the word of lane `lane` in column kk of batch b: run j of this warp
    // (4 words), runs dealt round-robin over the warps
    auto word_of = [&](int b, int kk) {
        const int j = (b * kGroup + kk) * 8 + (lane / 4);
        return (gw + j * kW) * 4 + (lane % 4);
    };
    int b = st.g0;
    for (;; ++b) {
        if (!st.loaded) {
            if ((gw + b * kGroup * 8 * kW) * 4 >= v.W) break;
            uint32_t wds[kGroup];
#pragma unroll
            for (int kk = 0; kk < kGroup; ++kk) {
                const int wi = word_of(b, kk);
                wds[kk] = wi < v.W ? v.bcur[wi] : 0u;
            }
#pragma unroll
            for (int kk = 0; kk < kGroup; ++kk) {
                const int wi = word_of(b, kk);
                if (wds[kk]) v.bcur[wi] = 0u;
                wb[kk * 32 + lane] = wds[kk];
            }
            __syncwarp();
            st.loaded = 1;
            st.kk = 0;
        }
        for (int kk = st.kk; kk < kGroup; ++kk) {
            // full rounds first, so that one more column always fits the list
            while (st.cnt >= 32) {
                if (st.n_slow > kQueue - 32) {
                    st.g0 = b;
                    st.kk = kk;
                    st.finished = 0;
                    return st;
                }
                const int t = list[st.cnt - 32 + lane];
                __syncwarp();
                st.cnt -= 32;
                round(t, true);
            }
            uint32_t w = wb[kk * 32 + lane];
            if (__any_sync(kAll, w != 0u)) {
                const uint32_t c = (uint32_t)__popc(w);
                uint32_t inc = c;
#pragma unroll
                for (int dd = 1; dd < 32; dd <<= 1) {
                    const uint32_t y = __shfl_up_sync(kAll, inc, dd);
                    if (lane >= dd) inc += y;
                }
                const int total = (int)__shfl_sync(kAll, inc, 31);
                int at = st.cnt + (int)(inc - c);
                const int base = word_of(b, kk) * 32;
                while (w) {
                    const int bit = __ffs(w) - 1;
                    list[at++] = base + bit;
                    w &= w - 1u;
                }
                __syncwarp();
                st.cnt += total;
                st.done += (unsigned long long)total;
            }
        }
        st.loaded = 0;
        st.kk = 0;
    }
    // the rest of the list, in rounds of up to 32
    while (st.cnt > 0) {
        if (st.n_slow > kQueue - 32) {
            st.g0 = b;
            st.finished = 0;
            return st;
        }
        const int n = st.cnt < 32 ? st.cnt : 32;
        const int t = lane < n ? list[st.cnt - n + lane] : 0;
        __syncwarp();
        st.cnt -= n;
        round(t, lane < n);
    }
    st.g0 = b;
    st.finished = 1;
    return st;
}

// The deferred tets of one warp's queue (n of them), in rounds of 32, with
// the full per-tet step: reactions and the non-inlined samplers.
template <int SA, bool kReact, int kC>
__device__ __noinline__ uint32_t slow_pass(const SlotDesc* __restrict__ dp, const ModelParams* __restrict__ mpp, int q,
                                           uint32_t* err, int n, unsigned long long* mass_delta) {
    const SlotDesc& d = *dp;
    const ModelParams& mp = *mpp;
    const PeriodView<kC> v(d, q);
    const int lane = threadIdx.x & 31;
    const int32_t* slowq = s_slowq[threadIdx.x >> 5];
    uint32_t bad = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
        const bool live = k0 + lane < n;
        const int t = live ? slowq[k0 + lane] : 0;
        uint32_t heavy = 0;
        int32_t N[SA];
        int4 o[SA];
        int4 sr = make_int4(-1, -1, -1, -1);
        uint4 pre = make_uint4(0u, 0u, 0u, 0u);
        long long before = 0;
        if (live) {
            sr = d.packed ? *reinterpret_cast<const int4*>(d.packed + 2 * t) : d.m.src[t];
            if (v.use_packed) pre = d.packed[2 * t + 1];
#pragma unroll
            for (int s = 0; s < SA; ++s) {
                if (s >= v.S) break;
                int32_t* p = v.Ncur + ((int64_t)s * v.T + t) * v.cstride;
                N[s] = *p;
                *p = 0;
                if (N[s] < 0) {          // wrapped past 2^31-1 by the previous period's adds
                    bad |= kErrOverflow;
                    N[s] = 0;
                }
                before += N[s];
            }
            bad |= step_tet<SA, kReact, true>(d.m, mp, v.period, v.tau_k, v.tau_kf, d.seed, v.thr, t, v.S, N, o,
                                              &heavy, err, v.tstride, v.use_packed, pre);
        }
        warp_split<SA>(heavy, d.seed, v.period, t, live ? key_of(d.m, t) : 0, v.thr, v.T, N, o, v.tstride,
                       v.use_packed, pre);
        if (live) bad |= v.template scatter<SA, kReact>(d, mp, t, sr, N, o);
        if (kReact) {
            // net molecules made by this tet's reactions: all it keeps and
            // sends minus what it held
            long long delta = 0;
            if (live) {
                delta = -before;
#pragma unroll
                for (int s = 0; s < SA; ++s) {
                    if (s >= v.S) break;
                    delta += (long long)N[s] + o[s].x + o[s].y + o[s].z + o[s].w;
                }
            }
#pragma unroll
            for (int dd = 16; dd > 0; dd >>= 1) delta += __shfl_xor_sync(0xffffffffu, delta, dd);
            if (lane == 0 && delta != 0) atomicAdd(mass_delta, (unsigned long long)delta);
        }
    }
    __syncwarp();   // the queue is refilled by the next light pass
    return bad;
}

// One simulation per cluster of kC CTAs (kC = 1: per CTA).  The cluster's
// first CTA owns the work-item index; the others read it through distributed
// shared memory.  cluster.sync() (a hardware barrier) separates periods.
//
// The tets to visit in a period are the set bits of that period's bitmap
// (global memory, one bit per tet, one bitmap per period parity).  Each
// visited word is cleared for its next use; a tet that keeps or receives
// molecules sets its bit in the other parity's bitmap (an OR, which is
// idempotent, so no membership test and no list are needed).  At the end of
// a slice both bitmaps are zero.
//
// Count adds are fire-and-forget reductions.  A count that an add takes past
// 2^31-1 wraps negative and is reported when read (next period, or the check
// at the end of the slice); the molecule total of the simulation, tracked per
// period (the slow pass adds what reactions make or consume), is kept below
// 2^32 - 1 so that no count can wrap all the way round unseen.
template <int SA, bool kReact, int kC>
__global__ void __launch_bounds__(kRunBlock, 1)
k_engine_run(const SlotDesc* __restrict__ descs, const ModelParams* __restrict__ mps, const int32_t* __restrict__ order,
             int32_t n_items, int32_t* head, uint32_t* err, unsigned long long* processed,
             unsigned long long* times) {
    namespace cg = cooperative_groups;
    constexpr unsigned kAll = 0xffffffffu;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = kC > 1 ? (int)cluster.block_rank() : 0;
    int32_t* item = kC > 1 ? cluster.map_shared_rank(&s_item, 0) : &s_item;
    unsigned long long* mass = kC > 1 ? cluster.map_shared_rank(&s_mass[0], 0) : &s_mass[0];
    auto csync = [&]() {
        if (kC > 1) cluster.sync();
        else __syncthreads();
    };
    const int lane = threadIdx.x & 31;
    unsigned long long done = 0;
    for (;;) {
        csync();
        if (rank == 0 && threadIdx.x == 0) {
            *item = atomicAdd(head, 1);
            mass[0] = mass[1] = mass[2] = 0ull;
        }
        csync();
        const int32_t k = *item;
        // every CTA has read the item before the leader may overwrite it or
        // any CTA leaves (a CTA's shared memory must outlive remote reads)
        csync();
        if (k >= n_items) break;
        const int slot = order[k];
        if (times && rank == 0 && threadIdx.x == 0) {
            times[4 * slot] = globaltimer_ns();
            times[4 * slot + 2] = 0ull;
        }
        unsigned long long item_done = 0;
        const SlotDesc& d = descs[slot];   // read-only; fields are loaded where used
        const ModelParams& mp = mps[slot];
        const int T = d.m.T;
        const int S = d.S;
        const int W = (T + 31) >> 5;
        const bool inter = d.N2 != nullptr;   // one species, interleaved counts
        uint32_t bad = 0;
        // initial bitmap: occupied tets and tets with a zero-order reaction on
        // (whole words, written by the first lane of each 32-tet run); and the
        // simulation's molecule total
        unsigned long long mine = 0;
        for (int base = rank * kRunBlock; base < W * 32; base += kC * kRunBlock) {
            const int t = base + threadIdx.x;
            bool occ = false;
            if (t < T) {
                occ = kReact && zero_order_on(d, mp, t);
                for (int s = 0; s < S; ++s) {
                    const int32_t c = d.N[0][(int64_t)s * T + t];
                    occ = occ || c > 0;
                    mine += (uint32_t)max(c, 0);
                    if (c < 0) bad |= kErrNegative;
                    if (inter) reinterpret_cast<int2*>(d.N2)[t] = make_int2(c, 0);
                }
            }
            const uint32_t word = __ballot_sync(kAll, occ);
            if (lane == 0 && (t >> 5) < W) d.bits[0][t >> 5] = word;
        }
#pragma unroll
        for (int dd = 16; dd > 0; dd >>= 1) mine += __shfl_xor_sync(kAll, mine, dd);
        if (lane == 0 && mine) atomicAdd(&mass[0], mine);
        // The molecule total after a period, kept below 2^32 - 1: then no
        // int32 count can wrap past 2^32 unseen (see PeriodView::scatter).
        // Reactions change it; the slow pass adds their net change.
        auto account = [&](int q) {
            if (rank == 0 && threadIdx.x == 0) {
                unsigned long long* dq = &mass[1 + (q & 1)];
                mass[0] += *dq;
                *dq = 0ull;
                if ((long long)mass[0] >= 4294967295ll) atomicOr(err, kErrOverflow);
            }
        };
        for (int q = d.q0; q < d.q1; ++q) {
            csync();   // the previous period's adds and bits are complete
            if (q > d.q0) account(q - 1);
            LightState st{0u, 0, 0, 0, 0, 0, 0, 0ull};
            for (;;) {
                st = light_pass<SA, kReact, kC>(descs + slot, mps + slot, q, err, st);
                bad |= st.bad;
                item_done += st.done;
                if (st.n_slow > 0)
                    bad |= slow_pass<SA, kReact, kC>(descs + slot, mps + slot, q, err, st.n_slow, &mass[1 + (q & 1)]);
                if (st.finished) break;
            }
        }
        csync();   // every add of the slice is complete
        account(d.q1 - 1);
        // a count the last period's adds took past 2^31-1 reads negative
        {
            const int half = (d.q1 - d.q0) & 1;
            for (int t = rank * kRunBlock + threadIdx.x; t < T; t += kC * kRunBlock) {
                if (inter) {
                    // the slice's counts are in the pairs' half (q1 - q0) & 1;
                    // hand them back in N[0]
                    const int32_t c = d.N2[2 * t + half];
                    if (c < 0) bad |= kErrOverflow;
                    d.N[0][t] = c;
                } else {
                    for (int s = 0; s < S; ++s)
                        if (d.N[half][(int64_t)s * T + t] < 0) bad |= kErrOverflow;
                }
            }
        }
        if (bad) atomicOr(err, bad);
        done += item_done;
        if (times) {
            if (lane == 0 && item_done) atomicAdd(times + 4 * slot + 2, item_done);
            if (rank == 0 && threadIdx.x == 0) times[4 * slot + 1] = globaltimer_ns();
        }
    }
    // entries processed: counted by lane 0 of each warp (warp-uniform)
    if (lane == 0 && done) atomicAdd(processed, done);
}

__global__ void k_pack(int32_t T, const int4* __restrict__ src, const uint4* __restrict__ thr, uint4* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int4 s4 = src[t];
    out[2 * t] = make_uint4((uint32_t)s4.x, (uint32_t)s4.y, (uint32_t)s4.z, (uint32_t)s4.w);
    out[2 * t + 1] = thr[t];
}

void launch_pack(int32_t T, const int4* src, const uint4* thr, uint4* out, cudaStream_t st) {
    k_pack<<<(T + 255) / 256, 256, 0, st>>>(T, src, thr, out);
    note_launch();
}

// Arguments of one engine launch.  `clusters` is the number of simulations
// to keep in flight (0: as many clusters as fit on the GPU at once); the
// launch never asks for more clusters than fit, since a persistent cluster
// that cannot be resident would only start when another one has finished.
struct EngineLaunch {
    const SlotDesc* descs;
    const ModelParams* mps;
    const int32_t* order;
    int32_t n_items;
    int32_t* head;
    uint32_t* err;
    unsigned long long* processed;
    unsigned long long* times;
    cudaStream_t st;
    int sms;
    int clusters;
    int used = 0;         // clusters launched
    int max_active = 0;   // clusters resident at once (occupancy query)
    bool query_only = false;   // fill max_active, launch nothing
};

template <int SA, bool R, int C>
cudaError_t launch_cluster(EngineLaunch& L) {
    auto kern = k_engine_run<SA, R, C>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmemBytes);
    if (ce != cudaSuccess) return ce;
    const size_t dyn = (size_t)kDynSmemBytes;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kRunBlock, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = L.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int fit = 0;
    if (C == 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRunBlock, dyn) == cudaSuccess)
            fit = per_sm * L.sms;
    } else if (cudaOccupancyMaxActiveClusters(&fit, kern, &cfg) != cudaSuccess) {
        fit = 0;
    }
    cudaGetLastError();
    if (fit <= 0) fit = std::max(1, L.sms / C);
    L.max_active = fit;
    if (L.query_only) return cudaSuccess;
    int n = L.clusters > 0 ? std::min(L.clusters, fit) : fit;
    n = std::max(1, std::min(n, L.n_items));
    L.used = n;
    if (C == 1) {
        kern<<<n, kRunBlock, dyn, L.st>>>(L.descs, L.mps, L.order, L.n_items, L.head, L.err, L.processed,
                                          L.times);
        return cudaGetLastError();
    }
    cfg.gridDim = dim3(n * C, 1, 1);
    return cudaLaunchKernelEx(&cfg, kern, L.descs, L.mps, L.order, L.n_items, L.head, L.err, L.processed,
                              L.times);
}

template <int SA>
cudaError_t launch_run_sa(bool react, int cluster, EngineLaunch& L) {
    if (cluster >= 8) return react ? launch_cluster<SA, true, 8>(L) : launch_cluster<SA, false, 8>(L);
    if (cluster == 4) return react ? launch_cluster<SA, true, 4>(L) : launch_cluster<SA, false, 4>(L);
    if (cluster == 2) return react ? launch_cluster<SA, true, 2>(L) : launch_cluster<SA, false, 2>(L);
    return react ? launch_cluster<SA, true, 1>(L) : launch_cluster<SA, false, 1>(L);
}

// Every instantiation of the engine kernel is launched once, with no work
// items, when the first engine is created on a device: each cluster takes an
// item index past the end and leaves, touching only the queue head (reset
// afterwards).  A step launches one kernel per species group on concurrent
// streams, and on the serving mix a step whose groups included kernels not
// launched before in the process ran the groups one after another (each
// started when the previous one ended) instead of side by side.
template <int SA, bool R, int C>
void warm_kernel(EngineLaunch& W) {
    if (launch_cluster<SA, R, C>(W) == cudaSuccess) note_launch();
    cudaGetLastError();   // a failure here shows again, and is reported, at a real launch
}

template <int SA>
void warm_kernels_sa(EngineLaunch& W) {
    warm_kernel<SA, false, 1>(W);
    warm_kernel<SA, true, 1>(W);
    warm_kernel<SA, false, 2>(W);
    warm_kernel<SA, true, 2>(W);
    warm_kernel<SA, false, 4>(W);
    warm_kernel<SA, true, 4>(W);
    warm_kernel<SA, false, 8>(W);
    warm_kernel<SA, true, 8>(W);
}

// head: int32[kGroups] of the engine being created (left zero); err and
// processed: its error word and entry counter (not written: no item runs).
void warm_engine_kernels(int32_t* head, uint32_t* err, unsigned long long* processed, int sms) {
    static std::mutex mu;
    static std::vector<int> warmed;   // devices done
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(warmed.begin(), warmed.end(), dev) != warmed.end()) return;
    EngineLaunch W{nullptr, nullptr, nullptr, 0, head, err, processed, nullptr, (cudaStream_t)0, sms, 1};
    warm_kernels_sa<1>(W);
    warm_kernels_sa<2>(W);
    warm_kernels_sa<4>(W);
    warm_kernels_sa<8>(W);
    warm_kernels_sa<kMaxS>(W);
    cudaMemsetAsync(head, 0, sizeof(int32_t) * 10, (cudaStream_t)0);
    cudaStreamSynchronize((cudaStream_t)0);
    cudaGetLastError();
    warmed.push_back(dev);
}

}  // namespace

struct rdsplit_engine {
    int32_t max_slots = 0;
    int64_t capacity = 0;
    cudaStream_t stream = 0;
    SlotDesc* d_desc = nullptr;
    ModelParams* d_mp = nullptr;
    int32_t* d_order = nullptr;
    int32_t* d_head = nullptr;
    uint32_t* err = nullptr;
    unsigned long long* processed = nullptr;  // (slot, tet) entries processed so far
    unsigned long long* d_times = nullptr;    // [max_slots][4] start, end (ns), entries of each slot's last slice
    int64_t launches = 0;                     // persistent launches issued
    int64_t steps = 0;                        // periods advanced, summed over step calls
    int32_t timing = 0;                       // time every launch with CUDA events
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double timing_ms = 0.0;
    int64_t timing_n = 0;
    int sms = 1;
    int32_t concurrency = 0;                  // simulations in flight (0 = as many as fit)
    int32_t last_in_flight = 0;               // clusters of the last launch
    int32_t last_max_active = 0;              // clusters that fit at once in the last launch
    int64_t slice_work = 0;                   // tet-periods per simulation and step call (0: no limit)
    int32_t last_groups = 0;                  // kernel groups of the last launch
    cudaStream_t aux[10] = {};                // one stream per kernel group
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[10] = {};
    int32_t cluster = 2;                      // CTAs per simulation (1, 2, 4 or 8)
    std::vector<rdsplit_mesh_t> slot_mesh;    // null = free
    std::vector<SlotDesc> h_desc;
    std::vector<int32_t> slot_q;              // local periods done
    std::vector<double> slot_t_end;
    std::vector<int32_t> finished;            // slots finished and not yet reported
    int64_t active_tets = 0;

    ~rdsplit_engine() {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (cudaEvent_t x : ev_join)
            if (x) cudaEventDestroy(x);
        for (cudaStream_t x : aux)
            if (x) cudaStreamDestroy(x);
        void* ps[] = {d_desc, d_mp, d_order, d_head, err, processed, d_times};
        for (void* p : ps) rdapi::dev_free(p);
    }
};

namespace {

int engine_err(rdsplit_engine* e, const char* where) {
    uint32_t v = 0;
    cudaError_t ce = cudaMemcpyAsync(&v, e->err, sizeof v, cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce));
    }
    if (v == 0) return RDSPLIT_OK;
    cudaMemsetAsync(e->err, 0, sizeof(uint32_t), e->stream);
    if (v & kErrOverflow) return rdapi::fail(RDSPLIT_EOVERFLOW, "%s: count overflow", where);
    if (v & kErrEventCap) return rdapi::fail(RDSPLIT_EOVERFLOW, "%s: SSA event cap exceeded", where);
    if (v & kErrNegative) return rdapi::fail(RDSPLIT_EINVAL, "%s: negative count", where);
    return rdapi::fail(RDSPLIT_ECUDA, "%s: device error bits 0x%x", where, v);
}

// Periods to reach t_end from t with Algorithm 1 (Step 1 aligns the last one)
// and the length of the last period.
void plan_periods(double t, double tau, double t_end, int64_t* P, double* tau_last, bool* last_short) {
    int64_t n = 0;
    *tau_last = tau;
    *last_short = false;
    while (t < t_end) {
        if (t + tau > t_end) {
            *tau_last = t_end - t;
            *last_short = true;
            t = t_end;
        } else {
            t = t + tau;
        }
        ++n;
    }
    *P = n;
}

void finish_slot(rdsplit_engine* e, int slot) {
    rdsplit_mesh* h = e->slot_mesh[slot];
    const SlotDesc& d = e->h_desc[slot];
    // a simulation added with t_end at or before its time ran no period and
    // keeps its time, as rdsplit_run would
    if (d.P > 0) h->t = e->slot_t_end[slot];
    h->period = (int64_t)d.period0 + d.P;
    e->active_tets -= h->T;
    e->slot_mesh[slot] = nullptr;
    e->finished.push_back(slot);
}

}  // namespace

extern "C" {

int rdsplit_engine_create(int32_t max_slots, int64_t max_active_tets, rdsplit_engine_t* out) {
    if (!out) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > (1 << 20)) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_create: bad max_slots");
    if (max_active_tets < 1) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_create: max_active_tets must be >= 1");
    rdsplit_engine* e = new rdsplit_engine();
    e->max_slots = max_slots;
    e->capacity = max_active_tets;
    e->d_desc = (SlotDesc*)rdapi::dev_alloc(sizeof(SlotDesc) * max_slots);
    e->d_mp = (ModelParams*)rdapi::dev_alloc(sizeof(ModelParams) * max_slots);
    e->d_order = (int32_t*)rdapi::dev_alloc(sizeof(int32_t) * max_slots);
    e->d_head = (int32_t*)rdapi::dev_alloc(sizeof(int32_t) * 10);
    e->err = (uint32_t*)rdapi::dev_alloc(sizeof(uint32_t));
    e->processed = (unsigned long long*)rdapi::dev_alloc(sizeof(unsigned long long));
    e->d_times = (unsigned long long*)rdapi::dev_alloc(sizeof(unsigned long long) * 4 * max_slots);
    if (!e->d_desc || !e->d_mp || !e->d_order || !e->d_head || !e->err || !e->processed || !e->d_times) {
        delete e;
        return rdapi::fail(RDSPLIT_ENOMEM, "rdsplit_engine_create: device allocation failed");
    }
    e->slot_mesh.assign(max_slots, nullptr);
    e->h_desc.assign(max_slots, SlotDesc{});
    e->slot_q.assign(max_slots, 0);
    e->slot_t_end.assign(max_slots, 0.0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev);
    warm_engine_kernels(e->d_head, e->err, e->processed, e->sms);
    if (cudaMemsetAsync(e->processed, 0, sizeof(unsigned long long), e->stream) != cudaSuccess ||
        cudaMemsetAsync(e->d_times, 0, sizeof(unsigned long long) * 4 * max_slots, e->stream) != cudaSuccess ||
        cudaMemsetAsync(e->err, 0, sizeof(uint32_t), e->stream) != cudaSuccess) {
        cudaGetLastError();
        delete e;
        return rdapi::fail(RDSPLIT_ECUDA, "rdsplit_engine_create: memset failed");
    }
    *out = e;
    return RDSPLIT_OK;
}

int rdsplit_engine_set_stream(rdsplit_engine_t e, void* stream) {
    if (!e) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_set_stream: NULL engine");
    e->stream = (cudaStream_t)stream;
    return RDSPLIT_OK;
}

int rdsplit_engine_add(rdsplit_engine_t e, rdsplit_mesh_t h, double t_end, uint64_t seed, int32_t* slot_out) {
    const char* where = "rdsplit_engine_add";
    if (!e || !h) return rdapi::fail(RDSPLIT_EINVAL, "%s: NULL argument", where);
    if (!h->has_model) return rdapi::fail(RDSPLIT_ESTATE, "%s: the mesh has no model", where);
    if (std::isnan(t_end)) return rdapi::fail(RDSPLIT_EINVAL, "%s: t_end is NaN", where);
    for (int s = 0; s < e->max_slots; ++s)
        if (e->slot_mesh[s] == h) return rdapi::fail(RDSPLIT_EINVAL, "%s: mesh already in the engine", where);
    int slot = -1;
    for (int s = 0; s < e->max_slots; ++s)
        if (!e->slot_mesh[s]) { slot = s; break; }
    if (slot < 0) return rdapi::fail(RDSPLIT_ENOMEM, "%s: no free slot", where);
    if (e->active_tets + h->T > e->capacity)
        return rdapi::fail(RDSPLIT_ENOMEM, "%s: active-tet capacity %lld exceeded", where, (long long)e->capacity);
    int64_t P = 0;
    double tau_last = h->tau;
    bool last_short = false;
    plan_periods(h->t, h->tau, t_end, &P, &tau_last, &last_short);
    if (h->period + P > (int64_t)0xffffffffll) return rdapi::fail(RDSPLIT_EOVERFLOW, "%s: period index exceeds 2^32-1", where);
    if (P > 0x7fffffffll) return rdapi::fail(RDSPLIT_EINVAL, "%s: too many periods", where);
    const size_t T = (size_t)h->T;
    const size_t W = (T + 31) / 32;
    if (!h->bits[0]) {
        h->bits[0] = (uint32_t*)rdapi::dev_alloc(4 * W);
        h->bits[1] = (uint32_t*)rdapi::dev_alloc(4 * W);
        if (!h->bits[0] || !h->bits[1]) return rdapi::fail(RDSPLIT_ENOMEM, "%s: bitmap allocation failed", where);
    }
    cudaStream_t st = e->stream;
    cudaError_t ce = cudaMemsetAsync(h->bits[0], 0, 4 * W, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->bits[1], 0, 4 * W, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->rem, 0, sizeof(int32_t) * T * h->S, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: memset failed: %s", where, cudaGetErrorString(ce));
    }
    if (last_short) launch_thresholds(h->T, h->mp, h->g, h->G, tau_last, h->thr_last, st);
    // one species without a zero-order reaction: packed per-tet records and
    // interleaved counts (fewer cache lines per active tet)
    bool zero = false;
    for (int r = 0; r < h->R; ++r) zero = zero || (h->mp.order[r] == 0 && h->mp.k[r] > 0.0);
    const bool pack = h->S == 1 && !zero && std::isfinite(h->tau);
    if (pack && !h->packed) {
        h->packed = (uint4*)rdapi::dev_alloc(32 * T);
        h->N2 = (int2*)rdapi::dev_alloc(8 * T);
        if (!h->packed || !h->N2) return rdapi::fail(RDSPLIT_ENOMEM, "%s: packed-record allocation failed", where);
    }
    if (pack) launch_pack(h->T, h->src, h->thr, h->packed, st);
    SlotDesc d{};
    d.m = h->dev_mesh();
    d.thr = h->thr;
    d.thr_last = last_short ? h->thr_last : h->thr;
    d.N[0] = h->cnt;
    d.N[1] = h->rem;
    d.bits[0] = h->bits[0];
    d.bits[1] = h->bits[1];
    d.packed = pack ? h->packed : nullptr;
    d.N2 = pack ? reinterpret_cast<int32_t*>(h->N2) : nullptr;
    d.seed = seed;
    d.period0 = (uint32_t)h->period;
    d.P = (int32_t)P;
    d.q0 = d.q1 = 0;
    d.last_short = last_short ? 1 : 0;
    d.S = h->S;
    d.zero_order = 0;
    for (int r = 0; r < h->R; ++r)
        if (h->mp.order[r] == 0 && h->mp.k[r] > 0.0) d.zero_order |= 1u << r;
    d.tau = h->tau;
    d.tau_last = tau_last;
    d.tauf = (float)h->tau;
    d.tau_lastf = (float)tau_last;
    ce = cudaMemcpyAsync(e->d_mp + slot, &h->mp, sizeof(ModelParams), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: model upload failed: %s", where, cudaGetErrorString(ce));
    }
    e->h_desc[slot] = d;
    e->slot_mesh[slot] = h;
    e->slot_q[slot] = 0;
    e->slot_t_end[slot] = t_end;
    e->active_tets += h->T;
    if (P == 0) finish_slot(e, slot);
    if (slot_out) *slot_out = slot;
    return RDSPLIT_OK;
}

// Advance every active simulation by up to n_steps periods in one persistent
// launch.  Finished handles receive their counts, time and period index;
// their slot ids are queued for rdsplit_engine_poll.
int rdsplit_engine_step(rdsplit_engine_t e, int64_t n_steps) {
    const char* where = "rdsplit_engine_step";
    if (!e) return rdapi::fail(RDSPLIT_EINVAL, "%s: NULL engine", where);
    if (n_steps <= 0) return RDSPLIT_OK;
    std::vector<int32_t> items;
    std::vector<double> work;
    int64_t max_adv = 0;
    for (int s = 0; s < e->max_slots; ++s) {
        rdsplit_mesh* h = e->slot_mesh[s];
        if (!h) continue;
        SlotDesc& d = e->h_desc[s];
        d.q0 = e->slot_q[s];
        // periods of this slice: n_steps, or fewer for a large simulation
        // when a work budget per slice is set (tets x periods), so that the
        // slices of one launch cost about the same
        int64_t n = n_steps;
        if (e->slice_work > 0) n = std::max<int64_t>(1, std::min<int64_t>(n_steps, e->slice_work / h->T));
        d.q1 = (int32_t)std::min<int64_t>((int64_t)d.P, (int64_t)d.q0 + n);
        if (d.q1 <= d.q0) continue;
        items.push_back(s);
        work.push_back((double)(d.q1 - d.q0) * (double)h->T * (double)h->S);
        max_adv = std::max<int64_t>(max_adv, d.q1 - d.q0);
    }
    if (items.empty()) return engine_err(e, where);
    // Simulations are launched in groups of one kernel instantiation each:
    // species class (1, 2, up to 4, up to 8, more) and with or without
    // reactions, so that a one-species simulation does not run the code
    // sized for eight.  Groups run concurrently on their own streams, the
    // resident clusters shared among them by work; largest first in each.
    auto cls_of = [&](int s) {
        const rdsplit_mesh* h = e->slot_mesh[s];
        const int S = h->S;
        const int c = S <= 1 ? 0 : (S <= 2 ? 1 : (S <= 4 ? 2 : (S <= 8 ? 3 : 4)));
        return 2 * c + (h->R > 0 ? 1 : 0);
    };
    constexpr int kGroups = 10;
    std::vector<size_t> idx(items.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
        const int ga = cls_of(items[a]), gb = cls_of(items[b]);
        return ga != gb ? ga < gb : work[a] > work[b];
    });
    std::vector<int32_t> order(items.size());
    int g_begin[kGroups + 1] = {0};
    double g_work[kGroups] = {0.0};
    int g_count[kGroups] = {0};
    for (size_t k = 0; k < idx.size(); ++k) {
        order[k] = items[idx[k]];
        const int g = cls_of(order[k]);
        g_count[g] += 1;
        g_work[g] += work[idx[k]];
    }
    for (int g = 0; g < kGroups; ++g) g_begin[g + 1] = g_begin[g] + g_count[g];
    int n_groups = 0;
    for (int g = 0; g < kGroups; ++g) n_groups += g_count[g] > 0 ? 1 : 0;
    cudaStream_t st = e->stream;
    cudaError_t ce = cudaMemcpyAsync(e->d_desc, e->h_desc.data(), sizeof(SlotDesc) * e->max_slots,
                                     cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(e->d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->d_head, 0, sizeof(int32_t) * kGroups, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: upload failed: %s", where, cudaGetErrorString(ce));
    }
    const int csize = e->cluster;
    if (e->timing && !e->ev[0]) {
        cudaEventCreate(&e->ev[0]);
        cudaEventCreate(&e->ev[1]);
    }
    if (e->timing) cudaEventRecord(e->ev[0], st);
    auto launch_group = [&](int g, EngineLaunch& L) -> cudaError_t {
        const bool react = (g & 1) != 0;
        switch (g >> 1) {
            case 0: return launch_run_sa<1>(react, csize, L);
            case 1: return launch_run_sa<2>(react, csize, L);
            case 2: return launch_run_sa<4>(react, csize, L);
            case 3: return launch_run_sa<8>(react, csize, L);
            default: return launch_run_sa<kMaxS>(react, csize, L);
        }
    };
    int used = 0, fit = 0;
    if (n_groups == 1) {
        int g = 0;
        while (g_count[g] == 0) ++g;
        // default: as many clusters as can be resident at once (one CTA per
        // SM where the GPCs allow it)
        EngineLaunch L{e->d_desc, e->d_mp, e->d_order, g_count[g], e->d_head, e->err, e->processed,
                       e->timing ? e->d_times : nullptr, st, e->sms, e->concurrency};
        ce = launch_group(g, L);
        used = L.used;
        fit = L.max_active;
    } else {
        // the clusters that fit, shared by work (at least one per group)
        EngineLaunch Q{e->d_desc, e->d_mp, e->d_order, 1, e->d_head, e->err, e->processed, nullptr, st, e->sms, 0};
        Q.query_only = true;
        ce = launch_group(7, Q);
        fit = Q.max_active;
        const int budget = e->concurrency > 0 ? std::min(e->concurrency, fit) : fit;
        double total = 0.0;
        for (int g = 0; g < kGroups; ++g) total += g_work[g];
        int share[kGroups] = {0};
        int given = 0;
        for (int g = 0; g < kGroups; ++g) {
            if (!g_count[g]) continue;
            share[g] = std::max(1, (int)((double)budget * g_work[g] / std::max(total, 1.0)));
            share[g] = std::min(share[g], g_count[g]);
            given += share[g];
        }
        while (given > std::max(budget, n_groups)) {   // trim the largest shares
            int gm = -1;
            for (int g = 0; g < kGroups; ++g)
                if (share[g] > 1 && (gm < 0 || share[g] > share[gm])) gm = g;
            if (gm < 0) break;
            share[gm] -= 1;
            given -= 1;
        }
        if (!e->ev_fork) {
            cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming);
            for (int g = 0; g < kGroups; ++g) {
                cudaStreamCreateWithFlags(&e->aux[g], cudaStreamNonBlocking);
                cudaEventCreateWithFlags(&e->ev_join[g], cudaEventDisableTiming);
            }
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e->ev_fork, st);
        for (int g = 0; g < kGroups && ce == cudaSuccess; ++g) {
            if (!g_count[g]) continue;
            ce = cudaStreamWaitEvent(e->aux[g], e->ev_fork, 0);
            EngineLaunch L{e->d_desc, e->d_mp, e->d_order + g_begin[g], g_count[g], e->d_head + g, e->err,
                           e->processed, e->timing ? e->d_times : nullptr, e->aux[g], e->sms, share[g]};
            if (ce == cudaSuccess) ce = launch_group(g, L);
            used += L.used;
            if (ce == cudaSuccess) ce = cudaEventRecord(e->ev_join[g], e->aux[g]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, e->ev_join[g], 0);
        }
    }
    EngineLaunch L{};
    L.used = used;
    L.max_active = fit;
    e->last_in_flight = L.used;
    e->last_max_active = L.max_active;
    e->last_groups = n_groups;
    if (e->timing) cudaEventRecord(e->ev[1], st);
    note_launch();
    e->launches += 1;
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: launch failed: %s", where, cudaGetErrorString(ce));
    }
    int rc = engine_err(e, where);
    if (e->timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e->ev[0], e->ev[1]) == cudaSuccess) {
            e->timing_ms += ms;
            e->timing_n += 1;
        }
        cudaGetLastError();
    }
    e->steps += max_adv;
    // the slice leaves each simulation's counts in N[(q1 - q0) & 1]
    for (int32_t s : items) {
        SlotDesc& d = e->h_desc[s];
        rdsplit_mesh* h = e->slot_mesh[s];
        if (((d.q1 - d.q0) & 1) && !d.N2) {
            std::swap(d.N[0], d.N[1]);
            std::swap(h->cnt, h->rem);
        }
        e->slot_q[s] = d.q1;
        if (d.q1 == d.P) finish_slot(e, s);
    }
    return rc;
}

int rdsplit_engine_poll(rdsplit_engine_t e, int32_t* slots, int32_t max, int32_t* n_out) {
    if (!e || !n_out) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_poll: NULL argument");
    int32_t n = 0;
    while (n < max && !e->finished.empty()) {
        slots[n++] = e->finished.front();
        e->finished.erase(e->finished.begin());
    }
    *n_out = n;
    return RDSPLIT_OK;
}

int rdsplit_engine_active(rdsplit_engine_t e, int32_t* n_slots, int64_t* n_tets) {
    if (!e) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_active: NULL engine");
    int32_t n = 0;
    for (int s = 0; s < e->max_slots; ++s) n += e->slot_mesh[s] ? 1 : 0;
    if (n_slots) *n_slots = n;
    if (n_tets) *n_tets = e->active_tets;
    return RDSPLIT_OK;
}

int rdsplit_engine_set_concurrency(rdsplit_engine_t e, int32_t in_flight, int32_t cluster) {
    if (!e || in_flight < 0 || !(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8))
        return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_set_concurrency: bad argument");
    e->concurrency = in_flight;
    e->cluster = cluster;
    return RDSPLIT_OK;
}

int rdsplit_engine_set_slice_work(rdsplit_engine_t e, int64_t max_tet_periods) {
    if (!e || max_tet_periods < 0) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_set_slice_work: bad argument");
    e->slice_work = max_tet_periods;
    return RDSPLIT_OK;
}

int rdsplit_engine_schedule(rdsplit_engine_t e, int32_t* in_flight, int32_t* cluster, int32_t* max_active) {
    if (!e) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_schedule: NULL engine");
    if (in_flight) *in_flight = e->last_in_flight;
    if (cluster) *cluster = e->cluster;
    if (max_active) *max_active = e->last_max_active;
    return RDSPLIT_OK;
}

int rdsplit_engine_set_timing(rdsplit_engine_t e, int32_t on) {
    if (!e || on < 0) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_set_timing: bad argument");
    e->timing = on;
    e->timing_ms = 0.0;
    e->timing_n = 0;
    return RDSPLIT_OK;
}

int rdsplit_engine_stats(rdsplit_engine_t e, int64_t* steps, int64_t* processed, double* timing_ms,
                         int64_t* timing_n) {
    if (!e) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_stats: NULL engine");
    unsigned long long p = 0;
    cudaError_t ce = cudaMemcpyAsync(&p, e->processed, sizeof p, cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "rdsplit_engine_stats: %s", cudaGetErrorString(ce));
    }
    if (steps) *steps = e->steps;
    if (processed) *processed = (int64_t)p;
    if (timing_ms) *timing_ms = e->timing_ms;
    if (timing_n) *timing_n = e->timing_n;
    return RDSPLIT_OK;
}

int rdsplit_engine_slot_times(rdsplit_engine_t e, int64_t* out, int32_t max_slots) {
    if (!e || !out || max_slots < 0)
        return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_engine_slot_times: bad argument");
    const int32_t n = std::min(max_slots, e->max_slots);
    std::vector<unsigned long long> buf(4 * (size_t)n);
    cudaError_t ce = cudaMemcpyAsync(buf.data(), e->d_times, sizeof(unsigned long long) * 4 * (size_t)n,
                                     cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    for (int32_t i = 0; ce == cudaSuccess && i < n; ++i)
        for (int k = 0; k < 3; ++k) out[3 * i + k] = (int64_t)buf[4 * i + k];
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "rdsplit_engine_slot_times: %s", cudaGetErrorString(ce));
    }
    return RDSPLIT_OK;
}

int rdsplit_engine_destroy(rdsplit_engine_t e) {
    if (!e) return RDSPLIT_OK;
    cudaStreamSynchronize(e->stream);
    delete e;
    return RDSPLIT_OK;
}

int rdsplit_ensemble_run(int32_t n, const rdsplit_mesh_t* meshes, const double* t_end, const uint64_t* seeds) {
    const char* where = "rdsplit_ensemble_run";
    if (n < 1 || !meshes || !t_end || !seeds) return rdapi::fail(RDSPLIT_EINVAL, "%s: bad arguments", where);
    int64_t tets = 0;
    for (int i = 0; i < n; ++i) {
        if (!meshes[i]) return rdapi::fail(RDSPLIT_EINVAL, "%s: NULL mesh %d", where, i);
        tets += meshes[i]->T;
    }
    rdsplit_engine_t e = nullptr;
    int rc = rdsplit_engine_create(n, tets, &e);
    if (rc) return rc;
    e->stream = meshes[0]->stream;
    for (int i = 0; i < n && rc == RDSPLIT_OK; ++i) rc = rdsplit_engine_add(e, meshes[i], t_end[i], seeds[i], nullptr);
    if (rc == RDSPLIT_OK) rc = rdsplit_engine_step(e, INT64_MAX / 4);
    rdsplit_engine_destroy(e);
    return rc;
}

}  // extern "C"
