// Host-side DVM generator of the C ABI: weights of a stencil from its
// velocities (Sect. III, Eq. defQua, defK, dimker), the lattice speed c* of
// a minimal DVM, and the wall augmentation of Sect. IV (Eq. 9.13, wallEq,
// defA).
//
// The null space of K(S) is the set of weight vectors whose Hermite moments
// of orders 1..Q all vanish (Eq. orth with n = 0; the argument below
// Eq. defK).  It is computed here from those moments directly, with one
// unknown per symmetry group (Eq. wdach): the matrix M has one row per
// Hermite tensor component (n_1..n_D) of order m <= Q, the product
// prod_d He_{n_d}(xi_d) summed over the group.  Its smallest singular value
// is linear in c - c*, where K's smallest eigenvalue is quadratic, so c* is
// located to rounding.  Singular values come from a one-sided Jacobi SVD.
#include <algorithm>
#include <array>
#include <cmath>
#include <limits>
#include <map>
#include <vector>

#include "lbm.h"

namespace {

constexpr double kNullRtol = 1e-9;     // singular value / largest: null direction
constexpr double kRootGap = 1e-9;      // accepted gap at a located c*
constexpr int kScan = 400;             // scan points of the c* search

struct Groups {
    std::vector<int> gid;     // group of each velocity
    std::vector<int> size;    // velocities per group
};

long factorial(int n) {
    long r = 1;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

// Groups of velocities related by component permutations and sign flips:
// equal multisets of absolute components.  LBM_EINVAL if an orbit is
// incomplete (the stencil is not closed under the lattice reflections).
int make_groups(int D, int V, const int* e, Groups& g) {
    std::map<std::array<int, 3>, int> ids;
    std::vector<std::array<int, 3>> keys;
    g.gid.assign(V, 0);
    for (int a = 0; a < V; ++a) {
        std::array<int, 3> k{0, 0, 0};
        for (int d = 0; d < D; ++d) k[d] = std::abs(e[a * D + d]);
        std::sort(k.begin(), k.begin() + D);
        auto it = ids.find(k);
        if (it == ids.end()) {
            it = ids.emplace(k, int(keys.size())).first;
            keys.push_back(k);
        }
        g.gid[a] = it->second;
    }
    g.size.assign(keys.size(), 0);
    for (int a = 0; a < V; ++a) ++g.size[g.gid[a]];
    for (size_t q = 0; q < keys.size(); ++q) {
        // orbit size: distinct permutations of the multiset x 2^(nonzero components)
        long perms = factorial(D);
        int nz = 0;
        for (int i = 0; i < D;) {
            int j = i;
            while (j < D && keys[q][j] == keys[q][i]) ++j;
            perms /= factorial(j - i);
            i = j;
        }
        for (int d = 0; d < D; ++d) nz += keys[q][d] != 0;
        if (long(g.size[q]) != perms * (1L << nz)) return LBM_EINVAL;
    }
    return LBM_OK;
}

double hermite(int n, double x) {       // probabilists' He_n
    double h0 = 1.0, h1 = x;
    if (n == 0) return h0;
    for (int k = 1; k < n; ++k) {
        const double h2 = x * h1 - k * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

// Column-major R x G matrix.
struct Mat {
    int R = 0, G = 0;
    std::vector<double> a;
    double& at(int r, int c) { return a[size_t(c) * R + r]; }
    double at(int r, int c) const { return a[size_t(c) * R + r]; }
};

// Orthogonality conditions per group, each order scaled by the norm of the
// same sums of absolute values, columns scaled to unit norm (colscale).
Mat moment_matrix(int D, int V, const int* e, const Groups& g, double c, int Q,
                  std::vector<double>& colscale) {
    const int G = int(g.size.size());
    std::vector<std::array<int, 3>> idx;
    std::vector<int> order;
    for (int m = 1; m <= Q; ++m)
        for (int n0 = m; n0 >= 0; --n0) {
            if (D == 2) {
                idx.push_back({n0, m - n0, 0});
                order.push_back(m);
            } else {
                for (int n1 = m - n0; n1 >= 0; --n1) {
                    idx.push_back({n0, n1, m - n0 - n1});
                    order.push_back(m);
                }
            }
        }
    Mat M;
    M.R = int(idx.size());
    M.G = G;
    M.a.assign(size_t(M.R) * G, 0.0);
    std::vector<double> A(size_t(M.R) * G, 0.0);     // sums of absolute values
    std::vector<std::array<double, 17>> he(size_t(V) * D);
    for (int a = 0; a < V; ++a)
        for (int d = 0; d < D; ++d)
            for (int n = 0; n <= Q; ++n) he[size_t(a) * D + d][n] = hermite(n, c * e[a * D + d]);
    for (int r = 0; r < M.R; ++r)
        for (int a = 0; a < V; ++a) {
            double v = 1.0;
            for (int d = 0; d < D; ++d) v *= he[size_t(a) * D + d][idx[r][d]];
            M.at(r, g.gid[a]) += v;
            A[size_t(g.gid[a]) * M.R + r] += std::fabs(v);
        }
    for (int r0 = 0; r0 < M.R;) {
        int r1 = r0;
        double s = 0.0;
        while (r1 < M.R && order[r1] == order[r0]) {
            for (int q = 0; q < G; ++q) s += A[size_t(q) * M.R + r1] * A[size_t(q) * M.R + r1];
            ++r1;
        }
        s = std::sqrt(s);
        for (int r = r0; r < r1; ++r)
            for (int q = 0; q < G; ++q) M.at(r, q) = s > 0 ? M.at(r, q) / s : 0.0;
        r0 = r1;
    }
    colscale.assign(G, 1.0);
    for (int q = 0; q < G; ++q) {
        double s = 0.0;
        for (int r = 0; r < M.R; ++r) s += M.at(r, q) * M.at(r, q);
        s = std::sqrt(s);
        colscale[q] = s > 0 ? s : 1.0;
        for (int r = 0; r < M.R; ++r) M.at(r, q) /= colscale[q];
    }
    return M;
}

// One-sided Jacobi SVD: U = M V with orthogonal columns; sigma_q = |U_q|,
// right singular vectors in the columns of Vr (G x G, column-major).
void jacobi_svd(Mat U, std::vector<double>& sigma, std::vector<double>& Vr) {
    const int R = U.R, G = U.G;
    Vr.assign(size_t(G) * G, 0.0);
    for (int q = 0; q < G; ++q) Vr[size_t(q) * G + q] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < G - 1; ++p)
            for (int q = p + 1; q < G; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = 0; r < R; ++r) {
                    al += U.at(r, p) * U.at(r, p);
                    be += U.at(r, q) * U.at(r, q);
                    ga += U.at(r, p) * U.at(r, q);
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-17 * std::sqrt(al * be)) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
                for (int r = 0; r < R; ++r) {
                    const double x = U.at(r, p), y = U.at(r, q);
                    U.at(r, p) = cs * x - sn * y;
                    U.at(r, q) = sn * x + cs * y;
                }
                for (int r = 0; r < G; ++r) {
                    double& x = Vr[size_t(p) * G + r];
                    double& y = Vr[size_t(q) * G + r];
                    const double xv = x, yv = y;
                    x = cs * xv - sn * yv;
                    y = sn * xv + cs * yv;
                }
            }
        if (!rotated) break;
    }
    sigma.assign(G, 0.0);
    for (int q = 0; q < G; ++q) {
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += U.at(r, q) * U.at(r, q);
        sigma[q] = std::sqrt(s);
    }
}

struct NullSpace {
    std::vector<std::vector<double>> basis;   // group weights (unscaled) per null direction
    double gap = 0.0;                         // smallest / largest singular value
};

NullSpace null_space(int D, int V, const int* e, const Groups& g, double c, int Q) {
    std::vector<double> colscale, sigma, Vr;
    const Mat M = moment_matrix(D, V, e, g, c, Q, colscale);
    jacobi_svd(M, sigma, Vr);
    const int G = M.G;
    const double smax = *std::max_element(sigma.begin(), sigma.end());
    NullSpace ns;
    ns.gap = *std::min_element(sigma.begin(), sigma.end()) / smax;
    for (int q = 0; q < G; ++q) {
        if (sigma[q] >= kNullRtol * smax) continue;
        std::vector<double> w(G);
        for (int r = 0; r < G; ++r) w[r] = Vr[size_t(q) * G + r] / colscale[r];
        ns.basis.push_back(w);
    }
    return ns;
}

// Velocity weights of a normalised (sum w = 1) group-weight vector.
bool expand_normalised(const Groups& g, const std::vector<double>& wg, int V, double* w) {
    double s = 0.0;
    for (size_t q = 0; q < wg.size(); ++q) s += g.size[q] * wg[q];
    if (!(std::fabs(s) > 0)) return false;
    for (int a = 0; a < V; ++a) w[a] = wg[g.gid[a]] / s;
    return true;
}

int check_args(int D, int V, const int* e, int Q) {
    if ((D != 2 && D != 3) || V < 1 || !e || Q < 1 || Q > 16) return LBM_EINVAL;
    return LBM_OK;
}

void nontrivial(int D, int Q, std::vector<std::array<int, 3>>& out) {
    out.clear();
    for (int n = 0; n <= Q; ++n)
        for (int mz = n; mz >= 0; --mz) {
            if (mz != 0 && !(mz & 1)) continue;
            for (int mx = n - mz; mx >= 0; --mx) {
                const int my = n - mz - mx;
                if ((mx & 1) || (my & 1) || my > mx) continue;
                if (D == 2 && my != 0) continue;
                out.push_back({mx, my, mz});
            }
        }
}

// Equilibrium wall moment over xi_z > 0 (Eq. Wscalar); 2D drops the y factor.
double wall_moment(int D, int mx, int my, int mz) {
    if ((mx & 1) || (my & 1)) return 0.0;
    const double pi = 3.14159265358979323846;
    const double gx = std::tgamma((mx + 1) / 2.0), gz = std::tgamma((mz + 1) / 2.0);
    if (D == 3)
        return std::pow(std::sqrt(2.0), mx + my + mz) / (8.0 * std::pow(std::sqrt(pi), 3)) * 4.0 *
               gx * std::tgamma((my + 1) / 2.0) * gz;
    if (my) return 0.0;
    return std::pow(std::sqrt(2.0), mx + mz) / (4.0 * pi) * 2.0 * gx * gz;
}

}  // namespace

extern "C" int lbm_dvm_solve_weights(int D, int V, const int* e, double c, int Q, double* w_out,
                                     int* nullity_out) {
    int rc = check_args(D, V, e, Q);
    if (rc) return rc;
    if (!w_out || !nullity_out || !(c > 0) || !std::isfinite(c)) return LBM_EINVAL;
    Groups g;
    if ((rc = make_groups(D, V, e, g))) return rc;
    const NullSpace ns = null_space(D, V, e, g, c, Q);
    *nullity_out = int(ns.basis.size());
    if (ns.basis.size() != 1 || !expand_normalised(g, ns.basis[0], V, w_out))
        for (int a = 0; a < V; ++a) w_out[a] = std::numeric_limits<double>::quiet_NaN();
    return LBM_OK;
}

extern "C" int lbm_dvm_find_c(int D, int V, const int* e, int Q, double c_lo, double c_hi,
                              double* c_out) {
    int rc = check_args(D, V, e, Q);
    if (rc) return rc;
    if (!c_out || !(c_lo > 0) || !(c_hi > c_lo) || !std::isfinite(c_hi)) return LBM_EINVAL;
    Groups g;
    if ((rc = make_groups(D, V, e, g))) return rc;
    auto gap = [&](double c) { return null_space(D, V, e, g, c, Q).gap; };
    std::vector<double> cs(kScan), f(kScan);
    for (int i = 0; i < kScan; ++i) {
        cs[i] = c_lo + (c_hi - c_lo) * i / (kScan - 1);
        f[i] = gap(cs[i]);
    }
    const double phi = (std::sqrt(5.0) - 1.0) / 2.0;
    std::vector<double> w(V);
    for (int i = 1; i < kScan - 1; ++i) {
        if (!(f[i] <= f[i - 1] && f[i] <= f[i + 1])) continue;
        double lo = cs[i - 1], hi = cs[i + 1];
        double x1 = hi - phi * (hi - lo), x2 = lo + phi * (hi - lo);
        double f1 = gap(x1), f2 = gap(x2);
        for (int it = 0; it < 200 && hi - lo > 4e-16 * hi; ++it) {
            if (f1 <= f2) {
                hi = x2;
                x2 = x1;
                f2 = f1;
                x1 = hi - phi * (hi - lo);
                f1 = gap(x1);
            } else {
                lo = x1;
                x1 = x2;
                f1 = f2;
                x2 = lo + phi * (hi - lo);
                f2 = gap(x2);
            }
        }
        const double c = 0.5 * (lo + hi);
        const NullSpace ns = null_space(D, V, e, g, c, Q);
        if (ns.gap > kRootGap || ns.basis.size() != 1) continue;
        if (!expand_normalised(g, ns.basis[0], V, w.data())) continue;
        if (std::all_of(w.begin(), w.end(), [](double x) { return x > 0; })) {
            *c_out = c;
            return LBM_OK;
        }
    }
    return LBM_ENOTCONV;
}

extern "C" int lbm_dvm_nontrivial_moments(int D, int Q, int cap, int* m_out, int* L_out) {
    if ((D != 2 && D != 3) || Q < 0 || Q > 16 || !L_out || cap < 0 || (cap > 0 && !m_out))
        return LBM_EINVAL;
    std::vector<std::array<int, 3>> mo;
    nontrivial(D, Q, mo);
    *L_out = int(mo.size());
    if (int(mo.size()) > cap) return m_out ? LBM_EINVAL : LBM_OK;
    for (size_t k = 0; k < mo.size(); ++k)
        for (int j = 0; j < 3; ++j) m_out[3 * k + j] = mo[k][j];
    return LBM_OK;
}

extern "C" int lbm_dvm_augment(int D, int V, const int* e, double c, int Q, int nk,
                               const int* k, double* w_out, double* residual_out) {
    int rc = check_args(D, V, e, Q);
    if (rc) return rc;
    if (!w_out || !(c > 0) || !std::isfinite(c) || nk < 0 || (nk > 0 && !k)) return LBM_EINVAL;
    std::vector<std::array<int, 3>> mo;
    nontrivial(D, Q, mo);
    for (int i = 0; i < nk; ++i)
        if (k[i] < 0 || k[i] >= int(mo.size())) return LBM_EINVAL;
    Groups g;
    if ((rc = make_groups(D, V, e, g))) return rc;
    const NullSpace ns = null_space(D, V, e, g, c, Q);
    const int J = int(ns.basis.size());
    if (J == 0) return LBM_EDEGREE;
    // rows: the selected wall moments over n.xi > 0 (Eq. defA), then sum w = 1
    Mat A;
    A.R = nk + 1;
    A.G = J;
    A.a.assign(size_t(A.R) * J, 0.0);
    std::vector<double> b(A.R, 0.0);
    for (int j = 0; j < J; ++j) {
        for (int a = 0; a < V; ++a) {
            const double wa = ns.basis[j][g.gid[a]];
            const double xx = c * e[a * D], xz = c * e[a * D + D - 1];
            const double xy = D == 3 ? c * e[a * D + 1] : 0.0;
            A.at(nk, j) += wa;
            if (!(xz > 0)) continue;
            for (int i = 0; i < nk; ++i) {
                const auto& m = mo[k[i]];
                A.at(i, j) += wa * std::pow(xx, m[0]) * (D == 3 ? std::pow(xy, m[1]) : 1.0) *
                              std::pow(xz, m[2]);
            }
        }
    }
    for (int i = 0; i < nk; ++i) b[i] = wall_moment(D, mo[k[i]][0], mo[k[i]][1], mo[k[i]][2]);
    b[nk] = 1.0;
    // least squares x = V S^+ U^T b from the Jacobi SVD (columns scaled to unit norm)
    std::vector<double> cn(J, 1.0);
    Mat As = A;
    for (int j = 0; j < J; ++j) {
        double s = 0.0;
        for (int r = 0; r < A.R; ++r) s += A.at(r, j) * A.at(r, j);
        cn[j] = s > 0 ? std::sqrt(s) : 1.0;
        for (int r = 0; r < A.R; ++r) As.at(r, j) /= cn[j];
    }
    std::vector<double> sigma, Vr;
    Mat U = As;
    jacobi_svd(As, sigma, Vr);
    // U = As Vr (columns U_q = sigma_q u_q)
    for (int q = 0; q < J; ++q)
        for (int r = 0; r < A.R; ++r) {
            double s = 0.0;
            for (int j = 0; j < J; ++j) s += As.at(r, j) * Vr[size_t(q) * J + j];
            U.at(r, q) = s;
        }
    const double smax = *std::max_element(sigma.begin(), sigma.end());
    std::vector<double> x(J, 0.0);
    for (int q = 0; q < J; ++q) {
        if (!(sigma[q] > 1e-13 * smax)) continue;
        double ub = 0.0;
        for (int r = 0; r < A.R; ++r) ub += U.at(r, q) * b[r];
        ub /= sigma[q] * sigma[q];
        for (int j = 0; j < J; ++j) x[j] += Vr[size_t(q) * J + j] * ub;
    }
    for (int j = 0; j < J; ++j) x[j] /= cn[j];
    double res = 0.0;
    for (int r = 0; r < A.R; ++r) {
        double s = -b[r];
        for (int j = 0; j < J; ++j) s += A.at(r, j) * x[j];
        res += s * s;
    }
    for (int a = 0; a < V; ++a) {
        double s = 0.0;
        for (int j = 0; j < J; ++j) s += x[j] * ns.basis[j][g.gid[a]];
        w_out[a] = s;
    }
    if (residual_out) *residual_out = std::sqrt(res);
    return LBM_OK;
}
