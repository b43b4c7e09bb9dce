// Host-side DVM utilities of the C ABI: group expansion (Eq. wdach), the
// (x, z) marginal of 3D sets, and the quadrature order (Eq. orth).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>
#include <vector>

#include "lbm.h"

namespace {

double gaussian_moment(int m) {  // (m-1)!! for even m, 0 for odd m
    if (m & 1) return 0.0;
    double r = 1.0;
    for (int k = m - 1; k > 0; k -= 2) r *= k;
    return r;
}

}  // namespace

extern "C" int lbm_dvm_expand(int D, int G, const int* reps, const int* vg, const double* wg,
                              int cap, int* e_out, double* w_out, int* V_out) {
    if ((D != 2 && D != 3) || G <= 0 || !reps || !wg || !e_out || !w_out || !V_out || cap < 0)
        return LBM_EINVAL;
    int V = 0;
    for (int g = 0; g < G; ++g) {
        std::array<int, 3> r{0, 0, 0};
        for (int d = 0; d < D; ++d) r[d] = reps[g * D + d];
        // orbit under permutations x sign flips (the reflections of the lattice)
        std::set<std::array<int, 3>> orbit;
        std::array<int, 3> perm{0, 1, 2};
        do {
            for (int signs = 0; signs < (1 << D); ++signs) {
                std::array<int, 3> v{0, 0, 0};
                for (int d = 0; d < D; ++d)
                    v[d] = ((signs >> d) & 1 ? -1 : 1) * r[perm[d]];
                orbit.insert(v);
            }
        } while (std::next_permutation(perm.begin(), perm.begin() + D));
        if (vg && vg[g] != (int)orbit.size()) return LBM_EINVAL;
        if (V + (int)orbit.size() > cap) return LBM_EINVAL;
        for (const auto& v : orbit) {
            for (int d = 0; d < D; ++d) e_out[V * D + d] = v[d];
            w_out[V] = wg[g];
            ++V;
        }
    }
    *V_out = V;
    return LBM_OK;
}

extern "C" int lbm_dvm_marginal_xz(int V3, const int* e3, const double* w3, int cap,
                                   int* e2_out, double* w2_out, int* V2_out) {
    if (V3 <= 0 || !e3 || !w3 || !e2_out || !w2_out || !V2_out) return LBM_EINVAL;
    std::map<std::pair<int, int>, double> acc;
    for (int a = 0; a < V3; ++a) acc[{e3[3 * a], e3[3 * a + 2]}] += w3[a];
    if ((int)acc.size() > cap) return LBM_EINVAL;
    int V = 0;
    for (const auto& kv : acc) {
        e2_out[2 * V] = kv.first.first;
        e2_out[2 * V + 1] = kv.first.second;
        w2_out[V] = kv.second;
        ++V;
    }
    *V2_out = V;
    return LBM_OK;
}

extern "C" int lbm_dvm_quadrature_order(const lbm_dvm* dvm, int* Q_out) {
    if (!dvm || !Q_out || dvm->D != 2 || dvm->V <= 0 || !dvm->e || !dvm->w) return LBM_EINVAL;
    int Q = -1;
    for (int deg = 0; deg <= 16; ++deg) {
        bool ok = true;
        for (int i = 0; i <= deg && ok; ++i) {
            const int j = deg - i;
            double sum = 0.0;
            for (int a = 0; a < dvm->V; ++a)
                sum += dvm->w[a] * std::pow(dvm->c * dvm->e[2 * a], i) *
                       std::pow(dvm->c * dvm->e[2 * a + 1], j);
            const double ref = gaussian_moment(i) * gaussian_moment(j);
            if (std::fabs(sum - ref) > 1e-9 * std::max(1.0, std::fabs(ref))) ok = false;
        }
        if (!ok) break;
        Q = deg;
    }
    *Q_out = Q;
    return LBM_OK;
}
