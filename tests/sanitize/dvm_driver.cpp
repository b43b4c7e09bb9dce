// Sanitizer run of the library's host-side DVM utilities (lbm_dvm_expand,
// lbm_dvm_marginal_xz, lbm_dvm_quadrature_order), including the error paths.
// Reads "D G" then G lines "rep... Vg wg" and c from stdin; prints V, the
// quadrature order of the 2D set (or of its (x, z) marginal) and the error
// codes of the boundary cases.
#include <cstdio>
#include <vector>

#include "lbm.h"

int main() {
    int D, G;
    double c;
    if (std::scanf("%d %d %lf", &D, &G, &c) != 3) return 2;
    std::vector<int> reps(G * D), vg(G);
    std::vector<double> wg(G);
    for (int g = 0; g < G; ++g) {
        for (int d = 0; d < D; ++d)
            if (std::scanf("%d", &reps[g * D + d]) != 1) return 2;
        if (std::scanf("%d %lf", &vg[g], &wg[g]) != 2) return 2;
    }
    int cap = 0;
    for (int v : vg) cap += v;
    std::vector<int> e(cap * D);
    std::vector<double> w(cap);
    int V = 0;
    int rc = lbm_dvm_expand(D, G, reps.data(), vg.data(), wg.data(), cap, e.data(), w.data(), &V);
    if (rc) return 4;
    // capacity one short must fail without writing past the buffers
    std::vector<int> e2((cap - 1) * D);
    std::vector<double> w2(cap - 1);
    int V2 = 0;
    const int rc_cap = lbm_dvm_expand(D, G, reps.data(), vg.data(), wg.data(), cap - 1, e2.data(),
                                      w2.data(), &V2);
    std::vector<int> e3;
    std::vector<double> w3;
    int Vq = V;
    if (D == 3) {
        e3.resize(2 * V);
        w3.resize(V);
        if (lbm_dvm_marginal_xz(V, e.data(), w.data(), V, e3.data(), w3.data(), &Vq)) return 5;
    } else {
        e3 = e;
        w3 = w;
    }
    lbm_dvm d{2, Vq, e3.data(), w3.data(), c};
    int Q = -1;
    if (lbm_dvm_quadrature_order(&d, &Q)) return 6;
    const int rc_null = lbm_dvm_quadrature_order(nullptr, &Q);
    std::printf("%d %d %d %d %d\n", V, Vq, Q, rc_cap, rc_null);
    return 0;
}
