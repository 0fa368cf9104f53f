// Host side of the C ABI declared in include/rdsplit.h: handle lifetime,
// argument validation, device memory, and the period loop of Algorithm 1
// (Step 1 alignment and Step 4 time advance, arXiv:1512.03126) around the
// kernels of rd_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rd_internal.h"
#include "rd_api_internal.h"
#include "rdsplit.h"

using namespace rdk;

namespace rdapi {

thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

static rdsplit_alloc_fn g_alloc = nullptr;
static rdsplit_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p) {
    if (!p) return;
    if (g_free) g_free(p, g_alloc_ctx);
    else cudaFree(p);
}

void set_allocator(rdsplit_alloc_fn a, rdsplit_free_fn f, void* ctx) {
    g_alloc = a;
    g_free = f;
    g_alloc_ctx = ctx;
}

}  // namespace rdapi

using namespace rdapi;

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(RDSPLIT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),     \
                        __FILE__, __LINE__);                                               \
        }                                                                                  \
    } while (0)

namespace {

template <typename T>
int alloc_into(T** p, size_t count, const char* what) {
    *p = (T*)dev_alloc(count * sizeof(T));
    if (!*p) return fail(RDSPLIT_ENOMEM, "device allocation of %s (%zu bytes) failed", what, count * sizeof(T));
    return RDSPLIT_OK;
}

// Read and clear the device error word; translate kernel error bits.
int check_err_impl(rdsplit_mesh* h, const char* where) {
    uint32_t e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, h->err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (e == 0) return RDSPLIT_OK;
    CUDA_TRY(cudaMemsetAsync(h->err, 0, sizeof(uint32_t), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (e & kErrAdjRange) return fail(RDSPLIT_EINVAL, "%s: neighbour index out of range or self-adjacent", where);
    if (e & kErrAdjAsym) return fail(RDSPLIT_EINVAL, "%s: adjacency is not symmetric", where);
    if (e & kErrVolume) return fail(RDSPLIT_EINVAL, "%s: a tet volume is not finite and positive", where);
    if (e & kErrFace) return fail(RDSPLIT_EINVAL, "%s: a face area or centroid distance is invalid", where);
    if (e & kErrOverflow) return fail(RDSPLIT_EOVERFLOW, "%s: a count exceeded INT32_MAX", where);
    if (e & kErrEventCap) return fail(RDSPLIT_EOVERFLOW, "%s: SSA event cap per tet and period exceeded", where);
    if (e & kErrNegative) return fail(RDSPLIT_EINVAL, "%s: negative count", where);
    return fail(RDSPLIT_ECUDA, "%s: device error bits 0x%x", where, e);
}

// Event pairs bracketing sampled period-kernel launches; collected after the
// stream is synchronised at the end of a run.
cudaEvent_t next_event(rdsplit_mesh* h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

void collect_timing(rdsplit_mesh* h) {
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]) == cudaSuccess) {
            h->timing_ms += ms;
            h->timing_n += 1;
        }
    }
    h->ev_used = 0;
    cudaGetLastError();
}

int launch_check(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RDSPLIT_ECUDA, "%s: kernel launch failed: %s", where, cudaGetErrorString(e));
    return RDSPLIT_OK;
}

}  // namespace

namespace rdapi {

int check_err(rdsplit_mesh* h, const char* where) { return check_err_impl(h, where); }

// The period loop of Algorithm 1 for one handle.  Step 1: the last period is
// shortened so that it ends on t_end.  Step 2-3 run in k_period, which also
// applies the previous period's transfers; the closing k_gather applies the
// last one.  Step 4: t += tau.
int run_loop(rdsplit_mesh* h, double t_end, int64_t max_periods, uint64_t seed) {
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "rdsplit_run: no model attached");
    if (std::isnan(t_end)) return fail(RDSPLIT_EINVAL, "rdsplit_run: t_end is NaN");
    DevMesh m = h->dev_mesh();
    DevState s = h->dev_state();
    const bool split = two_pass(h);
    const int block = period_block(h, sm_count());
    if (split && h->t < t_end && max_periods != 0) {
        cudaError_t ce = cudaMemsetAsync(h->dqn, 0, 2 * sizeof(int32_t), h->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(RDSPLIT_ECUDA, "rdsplit_run: %s", cudaGetErrorString(ce));
        }
    }
    int64_t j = 0;
    const int32_t* prev = nullptr;
    while (h->t < t_end && (max_periods < 0 || j < max_periods)) {
        if (h->period >= (int64_t)0xffffffffll)
            return fail(RDSPLIT_EOVERFLOW, "rdsplit_run: period index exceeds 2^32-1");
        double tau_k = h->tau;
        bool last = false;
        if (h->t + h->tau > t_end) {
            tau_k = t_end - h->t;
            last = true;
        }
        const uint4* thr = h->thr;
        if (last) {
            launch_thresholds(h->T, h->mp, h->g, h->G, tau_k, h->thr_last, h->stream);
            thr = h->thr_last;
        }
        int32_t* cur = h->inbox[j & 1];
        PeriodArgs a{(uint32_t)h->period, tau_k, (float)tau_k, seed, j == 0 ? 1 : 0, thr, prev, cur};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing_stride > 0 && j % h->timing_stride == 0) {
            e0 = next_event(h);
            e1 = next_event(h);
        }
        if (e0 && e1) cudaEventRecord(e0, h->stream);
        if (split) launch_period_split(m, h->mp, s, a, h->dq, h->dqn, (int32_t)(j & 1), block, h->stream);
        else launch_period(m, h->mp, s, a, block, h->stream);
        if (e0 && e1) cudaEventRecord(e1, h->stream);
        prev = cur;
        h->t = last ? t_end : h->t + h->tau;
        h->period += 1;
        j += 1;
    }
    if (j > 0) launch_gather(m, h->S, s, prev, h->stream);
    int rc = launch_check("rdsplit_run");
    if (rc) return rc;
    rc = check_err(h, "rdsplit_run");
    collect_timing(h);
    return rc;
}

}  // namespace rdapi

extern "C" {

const char* rdsplit_last_error(void) { return g_error.c_str(); }

int64_t rdsplit_kernel_launches(void) { return rdk::launches(); }

int rdsplit_set_allocator(rdsplit_alloc_fn a, rdsplit_free_fn f, void* ctx) {
    if ((a == nullptr) != (f == nullptr))
        return fail(RDSPLIT_EINVAL, "rdsplit_set_allocator: give both functions or neither");
    set_allocator(a, f, ctx);
    return RDSPLIT_OK;
}

}  // extern "C"

namespace {

// Spread the low 21 bits of x so that bit b lands on bit 3b.
uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Order of the tets along a Morton (Z-order) curve of their centroids:
// perm[i] = canonical id of the i-th tet on the curve (ties by id).  The box
// of the centroids is cut into 2^21 steps per axis.  Returns false if a
// centroid is not finite.
bool morton_order(int32_t T, const double* c, std::vector<int32_t>& perm) {
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int32_t t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            const double x = c[3 * (size_t)t + k];
            if (!std::isfinite(x)) return false;
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
    std::vector<std::pair<uint64_t, int32_t>> key((size_t)T);
    for (int32_t t = 0; t < T; ++t) {
        uint64_t m = 0;
        for (int k = 0; k < 3; ++k) {
            const double span = hi[k] - lo[k];
            double q = span > 0.0 ? (c[3 * (size_t)t + k] - lo[k]) / span * 2097151.0 : 0.0;
            q = std::min(std::max(q, 0.0), 2097151.0);
            m |= spread3((uint64_t)q) << k;
        }
        key[(size_t)t] = {m, t};
    }
    std::sort(key.begin(), key.end());
    perm.resize((size_t)T);
    for (int32_t i = 0; i < T; ++i) perm[(size_t)i] = key[(size_t)i].second;
    return true;
}

int mesh_create_impl(const char* where, int32_t n_tets, const int32_t* adj, const double* vol,
                     const double* face_area, const double* centroid_dist, const double* centroid, int32_t flags,
                     rdsplit_mesh_t* out) {
    if (!out) return fail(RDSPLIT_EINVAL, "%s: out is NULL", where);
    *out = nullptr;
    if (n_tets <= 0) return fail(RDSPLIT_EINVAL, "%s: n_tets must be > 0 (got %d)", where, n_tets);
    if (n_tets > (1 << 29)) return fail(RDSPLIT_EINVAL, "%s: n_tets too large", where);
    if (!adj || !vol || !face_area || !centroid_dist) return fail(RDSPLIT_EINVAL, "%s: NULL array", where);
    if (flags & ~RDSPLIT_REORDER_SFC) return fail(RDSPLIT_EINVAL, "%s: unknown flags 0x%x", where, flags);
    const bool reorder = (flags & RDSPLIT_REORDER_SFC) != 0;
    if (reorder && !centroid)
        return fail(RDSPLIT_EINVAL, "%s: RDSPLIT_REORDER_SFC needs the tet centroids (rdsplit_mesh_create_ex)", where);
    const size_t T = (size_t)n_tets;
    // stored order: canonical, or along the space-filling curve (the
    // arrays are permuted here; adjacency values are renumbered, invalid
    // ones passed through for the device-side validation to reject)
    std::vector<int32_t> perm, adj2;
    std::vector<double> vol2, area2, dist2;
    if (reorder) {
        if (!morton_order(n_tets, centroid, perm)) return fail(RDSPLIT_EINVAL, "%s: a centroid is not finite", where);
        std::vector<int32_t> inv(T);
        for (size_t i = 0; i < T; ++i) inv[(size_t)perm[i]] = (int32_t)i;
        adj2.resize(4 * T);
        vol2.resize(T);
        area2.resize(4 * T);
        dist2.resize(4 * T);
        for (size_t i = 0; i < T; ++i) {
            const size_t c = (size_t)perm[i];
            vol2[i] = vol[c];
            for (int f = 0; f < 4; ++f) {
                const int32_t u = adj[4 * c + f];
                adj2[4 * i + f] = (u >= 0 && u < n_tets) ? inv[(size_t)u] : u;
                area2[4 * i + f] = face_area[4 * c + f];
                dist2[4 * i + f] = centroid_dist[4 * c + f];
            }
        }
        adj = adj2.data();
        vol = vol2.data();
        face_area = area2.data();
        centroid_dist = dist2.data();
    }
    rdsplit_mesh* h = new rdsplit_mesh();
    h->T = n_tets;
    int32_t* d_adj = nullptr;
    double *d_area = nullptr, *d_dist = nullptr;
    int rc = RDSPLIT_OK;
    auto cleanup = [&](int code) {
        dev_free(d_adj);
        dev_free(d_area);
        dev_free(d_dist);
        if (code != RDSPLIT_OK) delete h;
        return code;
    };
    if ((rc = alloc_into(&d_adj, 4 * T, "adj")) || (rc = alloc_into(&d_area, 4 * T, "area")) ||
        (rc = alloc_into(&d_dist, 4 * T, "dist")) || (rc = alloc_into(&h->vol, T, "vol")) ||
        (rc = alloc_into(&h->src, T, "src")) || (rc = alloc_into(&h->g, 4 * T, "g")) ||
        (rc = alloc_into(&h->G, T, "G")) || (rc = alloc_into(&h->gmax, 1, "gmax")) ||
        (rc = alloc_into(&h->err, 1, "err")) || (reorder && (rc = alloc_into(&h->perm, T, "order"))))
        return cleanup(rc);
    cudaStream_t st = h->stream;
    cudaError_t ce = cudaSuccess;
    ce = ce ? ce : cudaMemcpyAsync(d_adj, adj, 16 * T, cudaMemcpyHostToDevice, st);
    ce = ce ? ce : cudaMemcpyAsync(h->vol, vol, 8 * T, cudaMemcpyHostToDevice, st);
    ce = ce ? ce : cudaMemcpyAsync(d_area, face_area, 32 * T, cudaMemcpyHostToDevice, st);
    ce = ce ? ce : cudaMemcpyAsync(d_dist, centroid_dist, 32 * T, cudaMemcpyHostToDevice, st);
    if (reorder) ce = ce ? ce : cudaMemcpyAsync(h->perm, perm.data(), 4 * T, cudaMemcpyHostToDevice, st);
    ce = ce ? ce : cudaMemsetAsync(h->gmax, 0, sizeof(unsigned long long), st);
    ce = ce ? ce : cudaMemsetAsync(h->err, 0, sizeof(uint32_t), st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(RDSPLIT_ECUDA, "%s: copy failed: %s", where, cudaGetErrorString(ce)));
    }
    launch_mesh_setup(n_tets, d_adj, h->vol, d_area, d_dist, h->src, h->g, h->G, h->gmax, h->err, st);
    if ((rc = launch_check(where))) return cleanup(rc);
    // the host arrays above are released on return: finish the copies first
    if ((rc = check_err(h, where))) return cleanup(rc);
    *out = h;
    return cleanup(RDSPLIT_OK);
}

}  // namespace

extern "C" {

int rdsplit_mesh_create(int32_t n_tets, const int32_t* adj, const double* vol, const double* face_area,
                        const double* centroid_dist, int32_t flags, rdsplit_mesh_t* out) {
    return mesh_create_impl("rdsplit_mesh_create", n_tets, adj, vol, face_area, centroid_dist, nullptr, flags, out);
}

int rdsplit_mesh_create_ex(int32_t n_tets, const int32_t* adj, const double* vol, const double* face_area,
                           const double* centroid_dist, const double* centroid, int32_t flags, rdsplit_mesh_t* out) {
    return mesh_create_impl("rdsplit_mesh_create_ex", n_tets, adj, vol, face_area, centroid_dist, centroid, flags,
                            out);
}

int rdsplit_get_order(rdsplit_mesh_t h, int32_t* perm) {
    if (!h || !perm) return fail(RDSPLIT_EINVAL, "rdsplit_get_order: NULL argument");
    if (!h->perm) {
        for (int32_t t = 0; t < h->T; ++t) perm[t] = t;
        return RDSPLIT_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(perm, h->perm, 4 * (size_t)h->T, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return RDSPLIT_OK;
}

int rdsplit_set_transfer_rule(rdsplit_mesh_t h, int32_t rule) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_transfer_rule: NULL handle");
    if (rule != RDSPLIT_TRANSFER_MEAN && rule != RDSPLIT_TRANSFER_END && rule != RDSPLIT_TRANSFER_MID)
        return fail(RDSPLIT_EINVAL, "rdsplit_set_transfer_rule: rule must be 0, 1 or 2");
    h->rule = rule;
    h->mp.rule = rule;
    return RDSPLIT_OK;
}

int rdsplit_set_zeta_outliers(rdsplit_mesh_t h, int32_t k) {
    const char* where = "rdsplit_set_zeta_outliers";
    if (!h) return fail(RDSPLIT_EINVAL, "%s: NULL handle", where);
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "%s: no model attached", where);
    if (k < 0 || k >= h->T) return fail(RDSPLIT_EINVAL, "%s: k must be in [0, n_tets)", where);
    cudaStream_t st = h->stream;
    unsigned long long* sel = nullptr;   // bits of the (k+1)-th largest G
    unsigned int* cnt = nullptr;
    int rc;
    if ((rc = alloc_into(&sel, 1, "selection")) || (rc = alloc_into(&cnt, 1, "count"))) {
        dev_free(sel);
        dev_free(cnt);
        return rc;
    }
    auto done = [&](int code) {
        dev_free(sel);
        dev_free(cnt);
        return code;
    };
    unsigned long long hi = 0;
    cudaError_t ce = cudaMemcpyAsync(&hi, h->gmax, sizeof hi, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    // largest x (as bits, G >= 0) with at least k+1 tets at or above it:
    // exactly the (k+1)-th largest G
    unsigned long long lo = 0;
    while (ce == cudaSuccess && lo < hi) {
        const unsigned long long mid = lo + (hi - lo + 1) / 2;
        unsigned int c = 0;
        ce = cudaMemsetAsync(cnt, 0, sizeof c, st);
        if (ce != cudaSuccess) break;
        launch_count_ge(h->T, h->G, mid, cnt, st);
        ce = cudaMemcpyAsync(&c, cnt, sizeof c, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) break;
        if (c >= (unsigned int)k + 1u) lo = mid;
        else hi = mid - 1;
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(sel, &lo, sizeof lo, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return done(fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce)));
    }
    launch_tau(h->D, h->S, sel, h->tau_scale, h->d_tau, st);
    ce = cudaMemcpyAsync(&h->tau, h->d_tau, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return done(fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce)));
    }
    if (std::isfinite(h->tau)) launch_thresholds(h->T, h->mp, h->g, h->G, h->tau, h->thr, st);
    if ((rc = launch_check(where))) return done(rc);
    h->outliers = k;
    return done(check_err(h, where));
}

int rdsplit_zeta_histogram(rdsplit_mesh_t h, int32_t nbins, int64_t* counts, double* mean, double* max_zeta) {
    const char* where = "rdsplit_zeta_histogram";
    if (!h || !counts) return fail(RDSPLIT_EINVAL, "%s: NULL argument", where);
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "%s: no model attached", where);
    if (nbins < 1 || nbins > (1 << 20)) return fail(RDSPLIT_EINVAL, "%s: nbins must be in 1..2^20", where);
    double dmax = 0.0;
    for (int s = 0; s < h->S; ++s) dmax = std::max(dmax, h->mp.D[s]);
    const double tau = std::isfinite(h->tau) ? h->tau : 0.0;
    cudaStream_t st = h->stream;
    unsigned long long* d_counts = nullptr;
    double* d_sum = nullptr;
    unsigned long long* d_max = nullptr;
    int rc;
    if ((rc = alloc_into(&d_counts, (size_t)nbins, "histogram")) || (rc = alloc_into(&d_sum, 1, "sum")) ||
        (rc = alloc_into(&d_max, 1, "max"))) {
        dev_free(d_counts);
        dev_free(d_sum);
        dev_free(d_max);
        return rc;
    }
    std::vector<unsigned long long> hc((size_t)nbins);
    double sum = 0.0;
    unsigned long long mb = 0;
    cudaError_t ce = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * nbins, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_sum, 0, sizeof(double), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), st);
    if (ce == cudaSuccess) {
        launch_zeta_hist(h->T, h->G, tau, dmax, nbins, d_counts, d_sum, d_max, st);
        ce = cudaMemcpyAsync(hc.data(), d_counts, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, st);
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&sum, d_sum, sizeof sum, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&mb, d_max, sizeof mb, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    dev_free(d_counts);
    dev_free(d_sum);
    dev_free(d_max);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce));
    }
    if ((rc = launch_check(where))) return rc;
    for (int b = 0; b < nbins; ++b) counts[b] = (int64_t)hc[b];
    if (mean) *mean = sum / (double)h->T;
    if (max_zeta) std::memcpy(max_zeta, &mb, sizeof(double));
    return RDSPLIT_OK;
}

int rdsplit_set_model(rdsplit_mesh_t h, int32_t S, const double* D, int32_t R, const int32_t* lhs,
                      const int32_t* rhs, const double* k, const uint8_t* mask, double tau_scale) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_model: NULL handle");
    if (S < 1 || S > RDSPLIT_MAX_SPECIES)
        return fail(RDSPLIT_EINVAL, "rdsplit_set_model: n_species must be in 1..%d", RDSPLIT_MAX_SPECIES);
    if (R < 0 || R > RDSPLIT_MAX_REACTIONS)
        return fail(RDSPLIT_EINVAL, "rdsplit_set_model: n_reactions must be in 0..%d", RDSPLIT_MAX_REACTIONS);
    if (!D) return fail(RDSPLIT_EINVAL, "rdsplit_set_model: D is NULL");
    if (R > 0 && (!lhs || !rhs || !k)) return fail(RDSPLIT_EINVAL, "rdsplit_set_model: reaction arrays NULL");
    if (!(tau_scale > 0.0) || !(tau_scale <= 1.0))
        return fail(RDSPLIT_EINVAL, "rdsplit_set_model: tau_scale must be in (0, 1]");
    ModelParams mp{};
    mp.S = S;
    mp.R = R;
    for (int s = 0; s < S; ++s) {
        if (!(D[s] >= 0.0) || !std::isfinite(D[s]))
            return fail(RDSPLIT_EINVAL, "rdsplit_set_model: D[%d] must be finite and >= 0", s);
        mp.D[s] = D[s];
    }
    for (int r = 0; r < R; ++r) {
        if (!(k[r] >= 0.0) || !std::isfinite(k[r]))
            return fail(RDSPLIT_EINVAL, "rdsplit_set_model: k[%d] must be finite and >= 0", r);
        mp.k[r] = k[r];
        int order = 0;
        for (int s = 0; s < S; ++s) {
            int a = lhs[r * S + s], b = rhs[r * S + s];
            if (a < 0 || b < 0 || a > 2 || b > 100)
                return fail(RDSPLIT_EINVAL, "rdsplit_set_model: bad stoichiometry in reaction %d", r);
            order += a;
            mp.lhs[r][s] = (int8_t)a;
            mp.delta[r][s] = (int8_t)(b - a);
        }
        if (order > 2) return fail(RDSPLIT_EINVAL, "rdsplit_set_model: reaction %d has order %d > 2", r, order);
        mp.order[r] = (int8_t)order;
    }
    mp.any_reaction = R > 0 ? 1 : 0;
    mp.has_mask = mask ? 1 : 0;
    mp.rule = h->rule;
    finish_model_params(mp);

    h->free_model();
    const size_t T = (size_t)h->T;
    int rc;
    if ((rc = alloc_into(&h->D, (size_t)S, "D")) || (rc = alloc_into(&h->d_tau, 1, "tau")) ||
        (rc = alloc_into(&h->cnt, T * S, "counts")) || (rc = alloc_into(&h->rem, T * S, "remainders")) ||
        (rc = alloc_into(&h->inbox[0], T * 4 * inbox_stride(S), "inboxes")) ||
        (rc = alloc_into(&h->inbox[1], T * 4 * inbox_stride(S), "inboxes")) ||
        (rc = alloc_into(&h->thr, T * S, "thresholds")) || (rc = alloc_into(&h->thr_last, T * S, "thresholds")) ||
        (rc = alloc_into(&h->staging, T * S, "staging")) || (rc = alloc_into(&h->avv, T, "avv")) ||
        (rc = alloc_into(&h->dq, T, "deferred-tet queue")) || (rc = alloc_into(&h->dqn, 2, "queue counters"))) {
        h->free_model();
        return rc;
    }
    cudaStream_t st = h->stream;
    if (mask) {
        uint8_t* d_m8 = nullptr;
        if ((rc = alloc_into(&d_m8, (size_t)R * T, "mask")) || (rc = alloc_into(&h->mask, T, "mask bits"))) {
            dev_free(d_m8);
            h->free_model();
            return rc;
        }
        cudaError_t ce = cudaMemcpyAsync(d_m8, mask, (size_t)R * T, cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess) launch_pack_mask(h->T, R, d_m8, h->mask, h->perm, st);
        cudaError_t ce2 = cudaStreamSynchronize(st);
        dev_free(d_m8);
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
            cudaGetLastError();
            h->free_model();
            return fail(RDSPLIT_ECUDA, "rdsplit_set_model: mask upload failed");
        }
    }
    CUDA_TRY(cudaMemcpyAsync(h->D, mp.D, sizeof(double) * S, cudaMemcpyHostToDevice, st));
    launch_avv(h->T, h->vol, h->avv, st);
    launch_tau(h->D, S, h->gmax, tau_scale, h->d_tau, st);
    CUDA_TRY(cudaMemcpyAsync(&h->tau, h->d_tau, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemsetAsync(h->cnt, 0, T * S * sizeof(int32_t), st));
    // boundary slots of the inboxes are never written and must read as zero
    CUDA_TRY(cudaMemsetAsync(h->inbox[0], 0, T * 4 * inbox_stride(S) * sizeof(int32_t), st));
    CUDA_TRY(cudaMemsetAsync(h->inbox[1], 0, T * 4 * inbox_stride(S) * sizeof(int32_t), st));
    CUDA_TRY(cudaMemsetAsync(h->rem, 0, T * S * sizeof(int32_t), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (std::isfinite(h->tau)) launch_thresholds(h->T, mp, h->g, h->G, h->tau, h->thr, st);
    if ((rc = launch_check("rdsplit_set_model"))) return rc;
    h->mp = mp;
    h->S = S;
    h->R = R;
    h->tau_scale = tau_scale;
    h->outliers = 0;
    h->has_model = true;
    h->t = 0.0;
    h->period = 0;
    return check_err(h, "rdsplit_set_model");
}

static int set_counts_impl(rdsplit_mesh_t h, const int32_t* counts, bool device) {
    if (!h || !counts) return fail(RDSPLIT_EINVAL, "rdsplit_set_counts: NULL argument");
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "rdsplit_set_counts: no model attached");
    const size_t n = (size_t)h->T * h->S;
    const int32_t* srcp = counts;
    if (!device) {
        CUDA_TRY(cudaMemcpyAsync(h->staging, counts, n * 4, cudaMemcpyHostToDevice, h->stream));
        srcp = h->staging;
    }
    launch_counts_in(h->T, h->S, srcp, h->cnt, h->err, h->perm, h->stream);
    int rc = launch_check("rdsplit_set_counts");
    if (rc) return rc;
    return check_err(h, "rdsplit_set_counts");
}

int rdsplit_set_counts(rdsplit_mesh_t h, const int32_t* counts) { return set_counts_impl(h, counts, false); }
int rdsplit_set_counts_device(rdsplit_mesh_t h, const int32_t* d) { return set_counts_impl(h, d, true); }

static int get_counts_impl(rdsplit_mesh_t h, int32_t* out, bool device) {
    if (!h || !out) return fail(RDSPLIT_EINVAL, "rdsplit_get_counts: NULL argument");
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "rdsplit_get_counts: no model attached");
    const size_t n = (size_t)h->T * h->S;
    int32_t* dst = device ? out : h->staging;
    launch_counts_out(h->T, h->S, h->cnt, dst, h->perm, h->stream);
    int rc = launch_check("rdsplit_get_counts");
    if (rc) return rc;
    if (!device) CUDA_TRY(cudaMemcpyAsync(out, h->staging, n * 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return RDSPLIT_OK;
}

int rdsplit_get_counts(rdsplit_mesh_t h, int32_t* out) { return get_counts_impl(h, out, false); }
int rdsplit_get_counts_device(rdsplit_mesh_t h, int32_t* d) { return get_counts_impl(h, d, true); }

int rdsplit_run(rdsplit_mesh_t h, double t_end, uint64_t seed) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_run: NULL handle");
    return run_loop(h, t_end, -1, seed);
}

int rdsplit_run_periods(rdsplit_mesh_t h, int64_t n_periods, uint64_t seed) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_run_periods: NULL handle");
    if (n_periods < 0) return fail(RDSPLIT_EINVAL, "rdsplit_run_periods: n_periods < 0");
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "rdsplit_run_periods: no model attached");
    if (!std::isfinite(h->tau)) return fail(RDSPLIT_EINVAL, "rdsplit_run_periods: no species diffuses");
    return run_loop(h, HUGE_VAL, n_periods, seed);
}

int rdsplit_get_time(rdsplit_mesh_t h, double* t, int64_t* period) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_get_time: NULL handle");
    if (t) *t = h->t;
    if (period) *period = h->period;
    return RDSPLIT_OK;
}

int rdsplit_set_time(rdsplit_mesh_t h, double t, int64_t period) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_time: NULL handle");
    if (!std::isfinite(t) || period < 0) return fail(RDSPLIT_EINVAL, "rdsplit_set_time: bad time or period");
    h->t = t;
    h->period = period;
    return RDSPLIT_OK;
}

int rdsplit_get_tau(rdsplit_mesh_t h, double* tau) {
    if (!h || !tau) return fail(RDSPLIT_EINVAL, "rdsplit_get_tau: NULL argument");
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "rdsplit_get_tau: no model attached");
    *tau = h->tau;
    return RDSPLIT_OK;
}

int rdsplit_get_shape(rdsplit_mesh_t h, int32_t* n_tets, int32_t* n_species) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_get_shape: NULL handle");
    if (n_tets) *n_tets = h->T;
    if (n_species) *n_species = h->S;
    return RDSPLIT_OK;
}

int rdsplit_set_stream(rdsplit_mesh_t h, void* stream) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_stream: NULL handle");
    h->stream = (cudaStream_t)stream;
    return RDSPLIT_OK;
}

int rdsplit_partition_set(rdsplit_mesh_t h, int32_t t0, int32_t t1) {
    const char* where = "rdsplit_partition_set";
    if (!h) return fail(RDSPLIT_EINVAL, "%s: NULL handle", where);
    if (h->perm) return fail(RDSPLIT_EINVAL, "%s: not available on a reordered mesh", where);
    if (t0 < 0 || t1 <= t0 || t1 > h->T) return fail(RDSPLIT_EINVAL, "%s: need 0 <= t0 < t1 <= n_tets", where);
    h->part_lo = t0;
    h->part_hi = t1;
    h->part_j = 0;
    return RDSPLIT_OK;
}

int rdsplit_partition_step(rdsplit_mesh_t h, double t_end, uint64_t seed, int32_t* more) {
    const char* where = "rdsplit_partition_step";
    if (!h) return fail(RDSPLIT_EINVAL, "%s: NULL handle", where);
    if (!h->has_model) return fail(RDSPLIT_ESTATE, "%s: no model attached", where);
    if (std::isnan(t_end)) return fail(RDSPLIT_EINVAL, "%s: t_end is NaN", where);
    if (h->part_hi <= h->part_lo) return fail(RDSPLIT_ESTATE, "%s: no partition set", where);
    if (h->t < t_end) {
        if (h->period >= (int64_t)0xffffffffll) return fail(RDSPLIT_EOVERFLOW, "%s: period index exceeds 2^32-1", where);
        double tau_k = h->tau;
        bool last = false;
        if (h->t + h->tau > t_end) {
            tau_k = t_end - h->t;
            last = true;
        }
        const uint4* thr = h->thr;
        if (last) {
            launch_thresholds(h->T, h->mp, h->g, h->G, tau_k, h->thr_last, h->stream);
            thr = h->thr_last;
        }
        const int64_t j = h->part_j;
        if (j == 0 && two_pass(h)) {
            CUDA_TRY(cudaMemsetAsync(h->dqn, 0, 2 * sizeof(int32_t), h->stream));
        }
        PeriodArgs a{(uint32_t)h->period, tau_k, (float)tau_k, seed, j == 0 ? 1 : 0, thr,
                     h->inbox[(j + 1) & 1], h->inbox[j & 1], h->part_lo, h->part_hi};
        const int block = period_block(h, sm_count());
        if (two_pass(h)) launch_period_split(h->dev_mesh(), h->mp, h->dev_state(), a, h->dq, h->dqn, (int32_t)(j & 1),
                                             block, h->stream);
        else launch_period(h->dev_mesh(), h->mp, h->dev_state(), a, block, h->stream);
        h->t = last ? t_end : h->t + h->tau;
        h->period += 1;
        h->part_j += 1;
        int rc = launch_check(where);
        if (rc) return rc;
        if ((rc = check_err(h, where))) return rc;
    }
    if (more) *more = h->t < t_end ? 1 : 0;
    return RDSPLIT_OK;
}

int rdsplit_partition_end(rdsplit_mesh_t h) {
    const char* where = "rdsplit_partition_end";
    if (!h) return fail(RDSPLIT_EINVAL, "%s: NULL handle", where);
    if (h->part_j > 0) {
        launch_gather(h->dev_mesh(), h->S, h->dev_state(), h->inbox[(h->part_j - 1) & 1], h->stream, h->part_lo,
                      h->part_hi);
        h->part_j = 0;
        int rc = launch_check(where);
        if (rc) return rc;
    }
    return check_err(h, where);
}

static int inbox_copy(rdsplit_mesh_t h, const int32_t* d_slots, int32_t n, int32_t* d_buf, bool out,
                      const char* where) {
    if (!h || (n > 0 && (!d_slots || !d_buf))) return fail(RDSPLIT_EINVAL, "%s: NULL argument", where);
    if (n < 0) return fail(RDSPLIT_EINVAL, "%s: n < 0", where);
    if (h->part_j == 0) return fail(RDSPLIT_ESTATE, "%s: no partition step since the last begin or end", where);
    int32_t* box = h->inbox[(h->part_j - 1) & 1];
    if (out) launch_inbox_export(h->S, box, d_slots, n, d_buf, h->stream);
    else launch_inbox_import(h->S, box, d_slots, n, d_buf, h->stream);
    int rc = launch_check(where);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return RDSPLIT_OK;
}

int rdsplit_inbox_export(rdsplit_mesh_t h, const int32_t* d_slots, int32_t n, int32_t* d_buf) {
    return inbox_copy(h, d_slots, n, d_buf, true, "rdsplit_inbox_export");
}

int rdsplit_inbox_import(rdsplit_mesh_t h, const int32_t* d_slots, int32_t n, const int32_t* d_buf) {
    return inbox_copy(h, d_slots, n, const_cast<int32_t*>(d_buf), false, "rdsplit_inbox_import");
}

int rdsplit_set_period_kernel(rdsplit_mesh_t h, int32_t mode, int32_t block) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_period_kernel: NULL handle");
    if (mode < 0 || mode > 2) return fail(RDSPLIT_EINVAL, "rdsplit_set_period_kernel: mode must be 0, 1 or 2");
    if (block != 0 && (block < 32 || block > 256 || block % 32))
        return fail(RDSPLIT_EINVAL, "rdsplit_set_period_kernel: block must be 0 or a multiple of 32 in 32..256");
    h->period_mode = mode;
    h->period_block = block;
    return RDSPLIT_OK;
}

int rdsplit_get_period_kernel(rdsplit_mesh_t h, int32_t* two_passes, int32_t* block) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_get_period_kernel: NULL handle");
    if (two_passes) *two_passes = two_pass(h) ? 1 : 0;
    if (block) *block = period_block(h, sm_count());
    return RDSPLIT_OK;
}

int rdsplit_set_timing(rdsplit_mesh_t h, int32_t stride) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_set_timing: NULL handle");
    if (stride < 0) return fail(RDSPLIT_EINVAL, "rdsplit_set_timing: stride < 0");
    h->timing_stride = stride;
    h->timing_ms = 0.0;
    h->timing_n = 0;
    return RDSPLIT_OK;
}

int rdsplit_get_timing(rdsplit_mesh_t h, double* total_ms, int64_t* n) {
    if (!h) return fail(RDSPLIT_EINVAL, "rdsplit_get_timing: NULL handle");
    if (total_ms) *total_ms = h->timing_ms;
    if (n) *n = h->timing_n;
    return RDSPLIT_OK;
}

int rdsplit_mesh_destroy(rdsplit_mesh_t h) {
    if (!h) return RDSPLIT_OK;
    cudaStreamSynchronize(h->stream);
    delete h;
    return RDSPLIT_OK;
}

}  // extern "C"
