// Host-side helpers and the handle layout shared by the C-ABI translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include "rd_internal.h"
#include "rdsplit.h"

namespace rdapi {
int fail(int code, const char* fmt, ...);
void* dev_alloc(size_t bytes);
void dev_free(void* p);
}  // namespace rdapi

// One mesh + model + state on the device.
struct rdsplit_mesh {
    int32_t T = 0, S = 0, R = 0;
    cudaStream_t stream = 0;
    // geometry
    int4* src = nullptr;
    double* g = nullptr;
    double* G = nullptr;
    double* vol = nullptr;
    uint32_t* mask = nullptr;
    float2* avv = nullptr;
    unsigned long long* gmax = nullptr;
    uint32_t* err = nullptr;
    int32_t* perm = nullptr;   // [T] canonical id of each stored tet (space-filling-curve order), or null
    // model and state
    double* D = nullptr;
    double* d_tau = nullptr;
    int32_t* cnt = nullptr;
    int32_t* rem = nullptr;
    int32_t* inbox[2] = {nullptr, nullptr};   // [T][4][Sp] transfer inboxes by period parity
    uint4* thr = nullptr;
    uint4* thr_last = nullptr;
    int32_t* staging = nullptr;
    uint32_t* bits[2] = {nullptr, nullptr};   // active-tet bitmaps by period parity (batched engine)
    uint4* packed = nullptr;   // one species: {reverse-face record, thresholds} per tet (batched engine)
    int2* N2 = nullptr;        // one species: {count, count} of two period parities (batched engine)
    int32_t* dq = nullptr;     // [T] tets deferred to the slow pass (two-pass period)
    int32_t* dqn = nullptr;    // [2] deferred-tet counters by period parity
    int32_t period_mode = 0;   // 0 auto (one pass), 1 one pass (k_period), 2 two passes (light + slow)
    int32_t period_block = 0;  // threads per block of the period kernel (0: by mesh size)
    int32_t part_lo = 0, part_hi = 0;  // partition steps advance stored tets [part_lo, part_hi)
    int64_t part_j = 0;                // periods done since the partition run began
    rdk::ModelParams mp{};
    bool has_model = false;
    int32_t rule = 0;          // transfer rule, kept across rdsplit_set_model
    double tau_scale = 1.0;    // of the attached model
    int32_t outliers = 0;      // fastest tets left out of the choice of tau
    // sampled kernel timing
    int32_t timing_stride = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double timing_ms = 0.0;
    int64_t timing_n = 0;
    double tau = 0.0;
    double t = 0.0;
    int64_t period = 0;

    rdk::DevMesh dev_mesh() const { return rdk::DevMesh{T, src, g, G, vol, mask, avv, perm}; }
    rdk::DevState dev_state() const { return rdk::DevState{cnt, rem, err}; }

    void free_model() {
        void* ps[] = {D, d_tau, cnt, rem, inbox[0], inbox[1], thr, thr_last, staging, mask, avv, dq, dqn};
        for (void* p : ps) rdapi::dev_free(p);
        D = nullptr; d_tau = nullptr; cnt = nullptr; rem = nullptr; inbox[0] = inbox[1] = nullptr;
        thr = nullptr; thr_last = nullptr; staging = nullptr; mask = nullptr; avv = nullptr;
        dq = nullptr; dqn = nullptr;
        has_model = false;
    }
    ~rdsplit_mesh() {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        free_model();
        void* ps[] = {src, g, G, vol, gmax, err, bits[0], bits[1], packed, N2, perm};
        for (void* p : ps) rdapi::dev_free(p);
    }
};


namespace rdapi {
// Whether the period loop of this handle runs in two passes (only when
// asked for: one pass measured faster on every workload here).
inline bool two_pass(const rdsplit_mesh* h) { return h->period_mode == 2; }

// Threads per block of the period kernel: as set, or 128 (measured fastest on
// the 2.4 M-tet bar: 310 us per period against 339 us with 256), smaller
// for a small mesh so that it still spreads over the SMs (at least 4 blocks
// per SM when the tets allow it; a power of two down to 32).
inline int period_block(const rdsplit_mesh* h, int sms) {
    if (h->period_block > 0) return h->period_block;
    int b = 128;
    while (b > 32 && (int64_t)h->T < (int64_t)4 * sms * b) b >>= 1;
    return b;
}
int run_loop(rdsplit_mesh* h, double t_end, int64_t max_periods, uint64_t seed);
int check_err(rdsplit_mesh* h, const char* where);
}  // namespace rdapi
