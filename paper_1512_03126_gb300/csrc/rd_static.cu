// rdsplit_run_static: the period loop of rdsplit_run for callers that must
// not allocate device memory.  All scratch (reverse-face table, face
// coefficients, thresholds, out-slots, remainders, the error word) lives in
// one file-scope static device array of RDSPLIT_STATIC_SCRATCH_BYTES; the
// caller passes the mesh, the model and the counts, and gets the counts back
// in place.  The kernels are the ones rdsplit_run launches, given pointers
// into that array.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "rd_api_internal.h"
#include "rd_internal.h"
#include "rdsplit.h"

using namespace rdk;

namespace {

// Every GPU that loads this library holds this array until the process exits.
// In host code, `g_static_scratch` is only a host-side stand-in for the device
// symbol, not a device address: a kernel handed it would fault (or, where the
// GPU can reach host memory, silently use the wrong memory).  Host code must
// use the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_static_scratch[RDSPLIT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int scratch_base(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "rdsplit_run_static: cudaGetDevice failed: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return rdapi::fail(RDSPLIT_ECUDA, "rdsplit_run_static: cudaGetSymbolAddress failed: %s",
                               cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return RDSPLIT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t err, gmax, tau, src, g, G, avv, mask, cnt, rem, out0, out1, thr, total;
};

Layout layout_for(size_t T, size_t S, bool masked) {
    Layout L{};
    size_t o = 0;
    L.err = o;  o += 256;
    L.gmax = o; o += 256;
    L.tau = o;  o += 256;
    L.src = o;  o = align256(o + 16 * T);
    L.g = o;    o = align256(o + 32 * T);
    L.G = o;    o = align256(o + 8 * T);
    L.avv = o;  o = align256(o + 8 * T);
    L.mask = o; o = align256(o + (masked ? 4 * T : 0));
    L.cnt = o;  o = align256(o + 4 * T * S);
    L.rem = o;  o = align256(o + 4 * T * S);
    L.out0 = o; o = align256(o + 16 * T * (size_t)inbox_stride((int32_t)S));
    L.out1 = o; o = align256(o + 16 * T * (size_t)inbox_stride((int32_t)S));
    L.thr = o;  o = align256(o + 16 * T * S);
    L.total = o;
    return L;
}

// tau from the model held in the kernel parameters (no device copy of D).
__global__ void k_static_tau(ModelParams mp, const unsigned long long* gmax_bits, double tau_scale, double* tau_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Gmax = __longlong_as_double((long long)*gmax_bits);
    double dmax = 0.0;
    for (int s = 0; s < mp.S; ++s) {
        double d = mp.D[s] * Gmax;
        if (d > dmax) dmax = d;
    }
    *tau_out = dmax > 0.0 ? tau_scale / dmax : __longlong_as_double(0x7ff0000000000000ll);
}

int model_params(int32_t S, const double* D, int32_t R, const int32_t* lhs, const int32_t* rhs, const double* k,
                 const uint8_t* mask, ModelParams* mp) {
    if (S < 1 || S > RDSPLIT_MAX_SPECIES)
        return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: n_species must be in 1..%d", RDSPLIT_MAX_SPECIES);
    if (R < 0 || R > RDSPLIT_MAX_REACTIONS)
        return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: n_reactions must be in 0..%d", RDSPLIT_MAX_REACTIONS);
    if (!D || (R > 0 && (!lhs || !rhs || !k))) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: NULL model array");
    *mp = ModelParams{};
    mp->S = S;
    mp->R = R;
    for (int s = 0; s < S; ++s) {
        if (!(D[s] >= 0.0) || !std::isfinite(D[s])) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: bad D[%d]", s);
        mp->D[s] = D[s];
    }
    for (int r = 0; r < R; ++r) {
        if (!(k[r] >= 0.0) || !std::isfinite(k[r])) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: bad k[%d]", r);
        mp->k[r] = k[r];
        int order = 0;
        for (int s = 0; s < S; ++s) {
            int a = lhs[r * S + s], b = rhs[r * S + s];
            if (a < 0 || b < 0 || a > 2 || b > 100)
                return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: bad stoichiometry in reaction %d", r);
            order += a;
            mp->lhs[r][s] = (int8_t)a;
            mp->delta[r][s] = (int8_t)(b - a);
        }
        if (order > 2) return rdapi::fail(RDSPLIT_EINVAL, "rdsplit_run_static: reaction %d has order > 2", r);
        mp->order[r] = (int8_t)order;
    }
    mp->any_reaction = R > 0 ? 1 : 0;
    mp->has_mask = mask ? 1 : 0;
    finish_model_params(*mp);
    return RDSPLIT_OK;
}

int read_err(unsigned char* base, const Layout& L, cudaStream_t st, const char* where) {
    uint32_t e = 0;
    cudaError_t ce = cudaMemcpyAsync(&e, base + L.err, sizeof e, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce));
    }
    if (e == 0) return RDSPLIT_OK;
    if (e & (kErrAdjRange | kErrAdjAsym | kErrVolume | kErrFace))
        return rdapi::fail(RDSPLIT_EINVAL, "%s: malformed mesh (error bits 0x%x)", where, e);
    if (e & (kErrOverflow | kErrEventCap)) return rdapi::fail(RDSPLIT_EOVERFLOW, "%s: count or event overflow", where);
    if (e & kErrNegative) return rdapi::fail(RDSPLIT_EINVAL, "%s: negative count", where);
    return rdapi::fail(RDSPLIT_ECUDA, "%s: device error bits 0x%x", where, e);
}

}  // namespace

extern "C" size_t rdsplit_static_scratch_bytes(int32_t n_tets, int32_t n_species, int32_t masked) {
    if (n_tets <= 0 || n_species <= 0) return 0;
    return layout_for((size_t)n_tets, (size_t)n_species, masked != 0).total;
}

extern "C" int rdsplit_run_static(int32_t n_tets, const int32_t* d_adj, const double* d_vol,
                                  const double* d_face_area, const double* d_centroid_dist, int32_t n_species,
                                  const double* D, int32_t n_reactions, const int32_t* lhs, const int32_t* rhs,
                                  const double* k, const uint8_t* d_rxn_tet_mask, double tau_scale,
                                  int32_t* d_counts, double* t, int64_t* period, double t_end, uint64_t seed,
                                  void* stream) {
    const char* where = "rdsplit_run_static";
    if (n_tets <= 0) return rdapi::fail(RDSPLIT_EINVAL, "%s: n_tets must be > 0", where);
    if (!d_adj || !d_vol || !d_face_area || !d_centroid_dist || !d_counts || !t || !period)
        return rdapi::fail(RDSPLIT_EINVAL, "%s: NULL argument", where);
    if (!(tau_scale > 0.0) || !(tau_scale <= 1.0)) return rdapi::fail(RDSPLIT_EINVAL, "%s: tau_scale must be in (0, 1]", where);
    if (std::isnan(t_end) || !std::isfinite(*t) || *period < 0) return rdapi::fail(RDSPLIT_EINVAL, "%s: bad time", where);
    ModelParams mp;
    int rc = model_params(n_species, D, n_reactions, lhs, rhs, k, d_rxn_tet_mask, &mp);
    if (rc) return rc;
    const size_t T = (size_t)n_tets, S = (size_t)n_species;
    Layout L = layout_for(T, S, d_rxn_tet_mask != nullptr);
    if (L.total > (size_t)RDSPLIT_STATIC_SCRATCH_BYTES)
        return rdapi::fail(RDSPLIT_EINVAL,
                           "%s: %d tets x %d species need %zu bytes of scratch; the static maximum is %zu "
                           "(RDSPLIT_STATIC_SCRATCH_BYTES)", where, n_tets, n_species, L.total,
                           (size_t)RDSPLIT_STATIC_SCRATCH_BYTES);
    unsigned char* base = nullptr;
    if ((rc = scratch_base(&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    uint32_t* err = (uint32_t*)(base + L.err);
    unsigned long long* gmax = (unsigned long long*)(base + L.gmax);
    double* d_tau = (double*)(base + L.tau);
    int4* src = (int4*)(base + L.src);
    double* g = (double*)(base + L.g);
    double* G = (double*)(base + L.G);
    float2* avv = (float2*)(base + L.avv);
    uint32_t* mask32 = d_rxn_tet_mask ? (uint32_t*)(base + L.mask) : nullptr;
    int32_t* cnt = (int32_t*)(base + L.cnt);
    int32_t* rem = (int32_t*)(base + L.rem);
    int32_t* out[2] = {(int32_t*)(base + L.out0), (int32_t*)(base + L.out1)};
    uint4* thr = (uint4*)(base + L.thr);

    // The array keeps the previous call's contents: clear what must start at
    // 0 (the control words, and both inboxes, whose boundary slots are never
    // written).
    cudaError_t ce = cudaMemsetAsync(base, 0, 3 * 256, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base + L.out0, 0, L.thr - L.out0, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: memset failed: %s", where, cudaGetErrorString(ce));
    }
    launch_mesh_setup(n_tets, d_adj, d_vol, d_face_area, d_centroid_dist, src, g, G, gmax, err, st);
    k_static_tau<<<1, 32, 0, st>>>(mp, gmax, tau_scale, d_tau);
    note_launch();
    if (mask32) launch_pack_mask(n_tets, n_reactions, d_rxn_tet_mask, mask32, nullptr, st);
    launch_avv(n_tets, d_vol, avv, st);
    double tau = 0.0;
    ce = cudaMemcpyAsync(&tau, d_tau, sizeof tau, cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return rdapi::fail(RDSPLIT_ECUDA, "%s: %s", where, cudaGetErrorString(ce));
    }
    if ((rc = read_err(base, L, st, where))) return rc;

    DevMesh m{n_tets, src, g, G, d_vol, mask32, avv, nullptr};
    DevState s{cnt, rem, err};
    launch_counts_in(n_tets, n_species, d_counts, cnt, err, nullptr, st);
    if (std::isfinite(tau)) launch_thresholds(n_tets, mp, g, G, tau, thr, st);

    // Algorithm 1: Step 1 aligns the last period to t_end, Steps 2-3 run in
    // the period kernel, Step 4 advances t.
    double tn = *t;
    int64_t pk = *period;
    int64_t j = 0;
    const int32_t* prev = nullptr;
    while (tn < t_end) {
        if (pk >= (int64_t)0xffffffffll) return rdapi::fail(RDSPLIT_EOVERFLOW, "%s: period index exceeds 2^32-1", where);
        double tau_k = tau;
        bool last = false;
        if (tn + tau > t_end) {
            tau_k = t_end - tn;
            last = true;
        }
        if (last) launch_thresholds(n_tets, mp, g, G, tau_k, thr, st);
        int32_t* cur = out[j & 1];
        PeriodArgs a{(uint32_t)pk, tau_k, (float)tau_k, seed, j == 0 ? 1 : 0, thr, prev, cur};
        launch_period(m, mp, s, a, 256, st);
        prev = cur;
        tn = last ? t_end : tn + tau;
        pk += 1;
        j += 1;
    }
    if (j > 0) launch_gather(m, n_species, s, prev, st);
    launch_counts_out(n_tets, n_species, cnt, d_counts, nullptr, st);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return rdapi::fail(RDSPLIT_ECUDA, "%s: launch failed: %s", where, cudaGetErrorString(ce));
    if ((rc = read_err(base, L, st, where))) return rc;
    *t = tn;
    *period = pk;
    return RDSPLIT_OK;
}
