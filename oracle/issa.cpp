// Brute-force exact spatial SSA (the paper's "ISSA", Sec. I and Sec. III):
// Gillespie's direct method over the whole mesh, every reaction in every tet
// and every single-molecule hop across every face being one event channel.
//
// TEST INFRASTRUCTURE ONLY: a statistical reference for small meshes
// (tens of tets).  It shares nothing with the operator-splitting oracle or the
// CUDA path but the problem definition: a molecule of species s in tet t
// hops to the neighbour across face f at rate D_s * A_tf / (V_t * dist_tf),
// and reactions follow mass action with the same unit conventions.
#include <cmath>
#include <cstdint>
#include <random>
#include <vector>

extern "C" int orc_issa_run(int32_t T, const int32_t* adj, const double* vol, const double* area,
                            const double* dist, int32_t S, const double* D, int32_t R,
                            const int32_t* lhs, const int32_t* rhs, const double* k,
                            const uint8_t* mask, int32_t* counts, double t_end, uint64_t seed) {
    const double NA = 6.02214076e23;
    std::mt19937_64 gen(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::vector<int64_t> N(counts, counts + (size_t)T * S);
    // hop rates per molecule
    std::vector<double> hop((size_t)T * S * 4, 0.0);
    for (int t = 0; t < T; ++t)
        for (int f = 0; f < 4; ++f) {
            if (adj[4 * t + f] < 0) continue;
            double geo = area[4 * t + f] / (vol[t] * dist[4 * t + f]);
            for (int s = 0; s < S; ++s) hop[((size_t)t * S + s) * 4 + f] = D[s] * geo;
        }
    // per-tet reaction constants
    std::vector<double> c((size_t)T * (R > 0 ? R : 1), 0.0);
    for (int t = 0; t < T; ++t)
        for (int r = 0; r < R; ++r) {
            int order = 0;
            for (int s = 0; s < S; ++s) order += lhs[r * S + s];
            double nv = NA * vol[t] * 1e3;
            double cr = order == 0 ? k[r] * nv : (order == 1 ? k[r] : k[r] / nv);
            if (mask && !mask[(size_t)r * T + t]) cr = 0.0;
            c[(size_t)t * R + r] = cr;
        }
    const size_t nd = (size_t)T * S * 4, nr = (size_t)T * R;
    std::vector<double> a(nd + nr);
    auto prop_react = [&](int t, int r) {
        double h = 1.0;
        for (int s = 0; s < S; ++s) {
            int nu = lhs[r * S + s];
            double n = (double)N[(size_t)t * S + s];
            if (nu == 1) h *= n;
            else if (nu == 2) h *= n * (n - 1.0) / 2.0;
        }
        return c[(size_t)t * R + r] * h;
    };
    double tnow = 0.0;
    for (;;) {
        double a0 = 0.0;
        for (int t = 0; t < T; ++t)
            for (int s = 0; s < S; ++s)
                for (int f = 0; f < 4; ++f) {
                    size_t i = ((size_t)t * S + s) * 4 + f;
                    a[i] = hop[i] * (double)N[(size_t)t * S + s];
                    a0 += a[i];
                }
        for (int t = 0; t < T; ++t)
            for (int r = 0; r < R; ++r) {
                a[nd + (size_t)t * R + r] = prop_react(t, r);
                a0 += a[nd + (size_t)t * R + r];
            }
        if (!(a0 > 0.0)) break;
        double u1 = 1.0 - U(gen);
        tnow += -std::log(u1) / a0;
        if (tnow >= t_end) break;
        double target = U(gen) * a0, cum = 0.0;
        size_t ev = a.size() - 1;
        for (size_t i = 0; i < a.size(); ++i) {
            cum += a[i];
            if (target < cum) { ev = i; break; }
        }
        while (a[ev] <= 0.0) --ev;
        if (ev < nd) {
            int f = (int)(ev % 4);
            size_t ts = ev / 4;
            int t = (int)(ts / S), s = (int)(ts % S);
            int u = adj[4 * t + f];
            N[(size_t)t * S + s] -= 1;
            N[(size_t)u * S + s] += 1;
        } else {
            size_t j = ev - nd;
            int t = (int)(j / R), r = (int)(j % R);
            for (int s = 0; s < S; ++s)
                N[(size_t)t * S + s] += rhs[r * S + s] - lhs[r * S + s];
        }
    }
    for (size_t i = 0; i < N.size(); ++i) counts[i] = (int32_t)N[i];
    return 0;
}
