// Internal interface between the host library (rd_api.cu) and the kernels
// (rd_kernels.cu).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rdk {

constexpr int kMaxS = 16;   // species
constexpr int kMaxR = 32;   // reactions (mask bits fit a uint32)

// Error bits raised by kernels into a device word.
enum : uint32_t {
    kErrAdjRange = 1u << 0,      // neighbour index out of range or self
    kErrAdjAsym = 1u << 1,       // adjacency not symmetric / duplicated
    kErrVolume = 1u << 2,        // volume not finite and positive
    kErrFace = 1u << 3,          // area or centroid distance invalid
    kErrNegative = 1u << 4,      // negative count (input or invariant)
    kErrOverflow = 1u << 5,      // a count would exceed INT32_MAX
    kErrEventCap = 1u << 6,      // more SSA events in one tet-period than the cap
};

// Chemistry, passed by value to kernels (lives in the constant bank).
struct ModelParams {
    int32_t S, R;
    int32_t has_mask;
    int32_t any_reaction;
    double D[kMaxS];
    double k[kMaxR];
    int8_t lhs[kMaxR][kMaxS];
    int8_t delta[kMaxR][kMaxS];   // rhs - lhs
    int8_t order[kMaxR];
    // For the single-precision "no event this period" pre-test: reactant
    // species (-1 = none; rs1 == rs2 for 2A), k as float, bits of k > 0.
    int8_t rs1[kMaxR], rs2[kMaxR];
    float kf[kMaxR];
    uint32_t kpos;
    // Per species: the reactions that consume it, and those that consume two
    // of it (2A): a reaction is possible in a tet unless a species it needs
    // is absent (or, for 2A, present only once).
    uint32_t needs[kMaxS];
    uint32_t needs2[kMaxS];
    // Transfer rule of the diffusion draw (Sec. II.C): kRuleMean (N-bar,
    // Eq. 3, the method), kRuleEnd (N at tau_k, first-order splitting) or
    // kRuleMid (N at tau_k / 2).
    int32_t rule;
};

constexpr int32_t kRuleMean = 0;
constexpr int32_t kRuleEnd = 1;
constexpr int32_t kRuleMid = 2;

// Fill the pre-test fields of a ModelParams whose lhs/k/order are set.
void finish_model_params(ModelParams& mp);

// Device arrays of one mesh + state.  Counts are species-major ([S][T]);
// inboxes are [T][4][Sp] (see PeriodArgs); src[t][f] = 4*adj[t][f] + (slot
// of t in that neighbour) or -1.
struct DevMesh {
    int32_t T;
    const int4* src;        // [T]
    const double* g;        // [T][4] face coefficient A/(V dist)
    const double* G;        // [T]   sum of g
    const double* vol;      // [T]
    const uint32_t* mask;   // [T]   reaction-on bits, or null
    const float2* avv;      // [T]   (N_A V_L, 1/(N_A V_L)) in single precision, or null
    const int32_t* perm;    // [T]   canonical id of each stored tet, or null (stored = canonical order)
};

// The canonical id of stored tet t, which keys its random streams.
__device__ __forceinline__ int key_of(const DevMesh& m, int t) { return m.perm ? __ldg(m.perm + t) : t; }

struct DevState {
    int32_t* cnt;           // [S][T] counts between runs
    int32_t* rem;           // [S][T] molecules that stayed in the last period
    uint32_t* err;          // error word
};

// ---- setup --------------------------------------------------------------
void launch_mesh_setup(int32_t T, const int32_t* adj, const double* vol, const double* area,
                       const double* dist, int4* src, double* g, double* G,
                       unsigned long long* gmax_bits, uint32_t* err, cudaStream_t st);
void launch_tau(const double* D, int32_t S, const unsigned long long* gmax_bits, double tau_scale,
                double* tau_out, cudaStream_t st);
void launch_thresholds(int32_t T, const ModelParams& mp, const double* g, const double* G, double tau_k,
                       uint4* thr, cudaStream_t st);
void launch_avv(int32_t T, const double* vol, float2* avv, cudaStream_t st);
void launch_count_ge(int32_t T, const double* G, unsigned long long xbits, unsigned int* count, cudaStream_t st);
void launch_zeta_hist(int32_t T, const double* G, double tau, double D, int32_t nbins, unsigned long long* counts,
                      double* sum, unsigned long long* maxbits, cudaStream_t st);
// perm: canonical id of each stored tet, or null (no reordering).
void launch_pack_mask(int32_t T, int32_t R, const uint8_t* mask8, uint32_t* mask32, const int32_t* perm,
                      cudaStream_t st);
void launch_counts_in(int32_t T, int32_t S, const int32_t* ts, int32_t* st_major, uint32_t* err,
                      const int32_t* perm, cudaStream_t st);
void launch_counts_out(int32_t T, int32_t S, const int32_t* st_major, int32_t* ts, const int32_t* perm,
                       cudaStream_t st);

// ---- one period (gather of the previous period fused with reactions and
// diffusion of this one) and the closing gather --------------------------
// Inboxes: int32 [T][4][Sp] with Sp = inbox_stride(S).  Slot [u][r] holds,
// per species, the molecules that the neighbour across face r of tet u sent
// to u in one period; a tet t writes its leavers through face f into slot
// src[t].f = 4 u + r of its neighbour u (each interior slot has exactly one
// writer per period, boundary slots are never written and stay zero), and
// reads its own four slots, contiguous, in the next period.
__host__ __device__ inline int32_t inbox_stride(int32_t S) { return S <= 2 ? S : (S + 3) & ~3; }

struct PeriodArgs {
    uint32_t period;        // global period index (random-stream key)
    double tau_k;           // length of this period
    float tau_kf;           // tau_k rounded to single precision
    uint64_t seed;
    int32_t first;          // 1: counts come from cnt (no pending transfer)
    const uint4* thr;       // [S][T] cumulative 32-bit face thresholds for tau_k
    const int32_t* in_prev; // [T][4][Sp] inboxes filled by the previous period
    int32_t* in_cur;        // [T][4][Sp] inboxes this period fills
    int32_t t_lo = 0;       // the period advances the stored tets [t_lo, t_hi) (a
    int32_t t_hi = 0;       // rank's range; 0, 0: all tets)
};
void launch_period(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a, int block,
                   cudaStream_t st);
void launch_gather(const DevMesh& m, int32_t S, const DevState& s, const int32_t* in_last, cudaStream_t st,
                   int32_t t_lo = 0, int32_t t_hi = 0);
// Copy inbox slots out of / into a packed buffer int32 [n][S] (the transfers
// across the cut faces of a partitioned mesh).
void launch_inbox_export(int32_t S, const int32_t* inbox, const int32_t* slots, int32_t n, int32_t* buf,
                         cudaStream_t st);
void launch_inbox_import(int32_t S, int32_t* inbox, const int32_t* slots, int32_t n, const int32_t* buf,
                         cudaStream_t st);
// The period in two passes (light pass, then the deferred tets): queue holds
// T entries, qcount two counters (both zero before the first period of a
// run; parity alternates 0, 1, 0, ... over the run's periods); `block` is the
// light pass's block size (32..256, a multiple of 32).
void launch_period_split(const DevMesh& m, const ModelParams& mp, const DevState& s, const PeriodArgs& a,
                         int32_t* queue, int32_t* qcount, int32_t parity, int block, cudaStream_t st);

int64_t launches();
int sm_count();       // multiprocessors of the current device
void note_launch();   // count a launch issued outside this file's launchers

}  // namespace rdk
