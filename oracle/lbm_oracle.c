/*
 * Oracle: plain fp64 CPU time stepping of the forced LB-BGK scheme with
 * diffuse Maxwell walls, for a 2D channel (x periodic, walls normal to y).
 *
 * TEST INFRASTRUCTURE ONLY.  The library never includes, links or calls this
 * file; only the tests, __graft_entry__.smoke() and the benchmark's
 * CPU-baseline leg load it.  It shares no code with the CUDA path.
 *
 * The code follows the paper's Sect. V (Numerical method) step by step, one
 * lattice node at a time, in the paper's order and notation:
 *
 *   state: fbar_a(x, y) before collision at time t (Eq. nm.7 defines fbar);
 *   (1) moments     rho = sum_a fbar_a,
 *                   rho u_i = sum_a fbar_a xi_ai + (dt/2) rho g_i   (Eq. nm.10)
 *   (2) equilibrium f0_a(rho, u), Hermite order N                    (Eq. nm.3,
 *                   and Eq. equi.hermite for the N = 4 term)
 *   (3) force       F_a (Eq. nm.4) with Pi the momentum flux of f, where
 *                   f = (2 tau fbar + dt feq)/(2 tau + dt) inverts Eq. nm.7
 *   (4) collision   fbar*_a = fbar_a - dt/(tau + dt/2) (fbar_a - feq_a),
 *                   feq_a = f0_a + tau F_a                   (Eq. nm.8, nm.2)
 *   (5) streaming   fbar_a(x, y, t+dt) = fbar*_a(x - e_ax, y - e_ay)
 *   (6) walls       populations whose source lies beyond a wall are set to
 *                   Psi rho_w w_a, Psi from the mass flux that left through
 *                   the wall in the same step (Eq. nm.14, nm.15).
 *
 * Lattice: node j sits half a spacing inside the walls (Sect. V, "as for the
 * half-way bounce-back scheme"); xi_a = c e_a with integer e_a, so one step
 * moves population a by e_a nodes.
 *
 * Readings of silent points (listed in the design notes):
 *  - walls act on fbar directly: the unknown fbar_a = Psi rho_w w_a, with Psi
 *    from the outgoing post-collision fbar* (the fbar form of Eq. nm.14 is
 *    not printed);
 *  - a population with |e_y| > 1 crosses the wall from each of the |e_y|
 *    rows nearest to it; all rows y < e_y of an incoming a are unknown;
 *  - an outgoing population is credited to the column it lands on,
 *    (x_source + e_x) mod Nx, so Psi is a per-column quantity;
 *  - the force term of Eq. nm.4 is used unchanged for N = 4 (behind
 *    force_a3 = 1, the variant with the fourth-order term of a^(3) = rho uuu);
 *  - behind wall_mode = 1, the alternative reading of the wall: the condition
 *    holds for f and fbar follows through Eq. nm.7 (transform_wall_nodes).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle.h"

static int wrap(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }

/* Index of population a at node (x, y): planes [V][Ny][Nx], x fastest. */
static long at(const oracle_params* p, int a, int x, int y) {
    return ((long)a * p->Ny + y) * p->Nx + x;
}

/* Equilibrium f0_a(rho, u) / (rho w_a), Eq. nm.3 for N <= 3; the N = 4 term
 * is (1/4!) u_i u_j u_k u_l H^(4)_ijkl(xi_a) of Eq. equi.hermite, which
 * contracts to (s^4 - 6 s^2 u^2 + 3 u^4)/24 with s = u.xi_a. */
static double f0_over_rho_w(int N, double s, double uu) {
    double r = 1.0 + s + 0.5 * (s * s - uu);
    if (N >= 3) r += s * (s * s - 3.0 * uu) / 6.0;
    if (N >= 4) r += (s * s * s * s - 6.0 * s * s * uu + 3.0 * uu * uu) / 24.0;
    return r;
}

/* H^(2)_ij(xi) = xi_i xi_j - delta_ij (Eq. defH). */
static double H2(const double xi[2], int i, int j) {
    return xi[i] * xi[j] - (i == j ? 1.0 : 0.0);
}

/* Body-force term F_a of Eq. nm.4 for velocity xi (w_a factored in). */
static double force_term(int N, int a3, double rho, const double u[2], const double g[2],
                         const double Pi[2][2], const double xi[2], double wa) {
    double gxi = g[0] * xi[0] + g[1] * xi[1];
    double uxi = u[0] * xi[0] + u[1] * xi[1];
    double ug = u[0] * g[0] + u[1] * g[1];
    double r = gxi + (gxi * uxi - ug);
    if (N >= 3) {
        double t = 0.0;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                t += (Pi[i][j] - (i == j ? rho : 0.0)) *
                     (gxi * H2(xi, i, j) - 2.0 * g[i] * xi[j]);
        r += t / (2.0 * rho);
    }
    if (N >= 4 && a3) {
        /* (1/3!) g_i a^(3)_jkl H^(4)_ijkl(xi) / rho with a^(3) = rho u u u:
         * H^(4) = xi^4 - 6 sym(xi xi delta) + 3 sym(delta delta) contracted
         * with g u u u gives the four terms below. */
        const double uu = u[0] * u[0] + u[1] * u[1];
        r += (gxi * uxi * uxi * uxi - 3.0 * gxi * uxi * uu - 3.0 * uxi * uxi * ug +
              3.0 * ug * uu) / 6.0;
    }
    return rho * wa * r;
}

/* Collision at one node, steps (1)-(4).  fin/fout hold the V populations. */
static void collide_node(const oracle_params* p, const double* fin, double* fout,
                         double* f0, double* F) {
    const int V = p->V;
    const double c = p->c, tau = p->tau, dt = p->dt;
    const double g[2] = {p->gx, p->gy};

    /* (1) moments, Eq. nm.10 */
    double rho = 0.0, mom[2] = {0.0, 0.0};
    for (int a = 0; a < V; ++a) {
        rho += fin[a];
        mom[0] += fin[a] * c * p->ex[a];
        mom[1] += fin[a] * c * p->ey[a];
    }
    double u[2];
    for (int i = 0; i < 2; ++i) u[i] = (mom[i] + 0.5 * dt * rho * g[i]) / rho;
    double uu = u[0] * u[0] + u[1] * u[1];

    /* (2) equilibrium, Eq. nm.3 */
    for (int a = 0; a < V; ++a) {
        double xi[2] = {c * p->ex[a], c * p->ey[a]};
        double s = u[0] * xi[0] + u[1] * xi[1];
        f0[a] = rho * p->w[a] * f0_over_rho_w(p->N, s, uu);
    }

    /* (3) Pi of f.  f = (2 tau fbar + dt feq)/(2 tau + dt) inverts Eq. nm.7.
     * feq depends on Pi only through the Pi term of Eq. nm.4, a third-order
     * Hermite term whose second moment vanishes by Eq. orth, so Pi is found
     * by evaluating feq once with Pi = rho delta (that term zero) and
     * summing sum_a f_a xi_ai xi_aj. */
    double Pi0[2][2] = {{rho, 0.0}, {0.0, rho}};
    double Pi[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int a = 0; a < V; ++a) {
        double xi[2] = {c * p->ex[a], c * p->ey[a]};
        double feq = f0[a] + tau * force_term(p->N, p->force_a3, rho, u, g, Pi0, xi, p->w[a]);
        double fa = (2.0 * tau * fin[a] + dt * feq) / (2.0 * tau + dt);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) Pi[i][j] += fa * xi[i] * xi[j];
    }
    for (int a = 0; a < V; ++a) {
        double xi[2] = {c * p->ex[a], c * p->ey[a]};
        F[a] = force_term(p->N, p->force_a3, rho, u, g, Pi, xi, p->w[a]);
    }

    /* (4) collision, Eq. nm.8 with feq = f0 + tau F (Eq. nm.2) */
    double omega = dt / (tau + 0.5 * dt);
    for (int a = 0; a < V; ++a) {
        double feq = f0[a] + tau * F[a];
        fout[a] = fin[a] - omega * (fin[a] - feq);
    }
}

/* Nodes are independent: the row loop may run in parallel (OpenMP build of
 * the CPU baseline only; each node's arithmetic is the same either way). */
int oracle_collide(const oracle_params* p, const double* f, double* fstar) {
    const int V = p->V;
    int failed = 0;
#pragma omp parallel reduction(| : failed)
    {
        double* fin = malloc(sizeof(double) * 4 * V);
        if (!fin) {
            failed = 1;
        } else {
            double *fout = fin + V, *f0 = fin + 2 * V, *F = fin + 3 * V;
#pragma omp for schedule(static)
            for (int y = 0; y < p->Ny; ++y)
                for (int x = 0; x < p->Nx; ++x) {
                    for (int a = 0; a < V; ++a) fin[a] = f[at(p, a, x, y)];
                    collide_node(p, fin, fout, f0, F);
                    for (int a = 0; a < V; ++a) fstar[at(p, a, x, y)] = fout[a];
                }
            free(fin);
        }
    }
    return failed ? -1 : 0;
}

/* Alternative reading of the wall condition (wall_mode = 1): Eq. nm.14 sets
 * the unknown f_a = Psi rho_w w_a, and fbar follows from f through Eq. nm.7
 * with the BGK operator and without the force term,
 *   fbar_a = f_a + (dt / 2 tau) (f_a - f0_a(rho, u)),
 * rho, u the node's moments (Eq. nm.10).  Those moments contain the unknowns
 * themselves, so each wall node is solved by fixed-point iteration, starting
 * from the plain values Psi rho_w w_a already in f (a contraction with factor
 * ~ dt / 2 tau).  Psi keeps its value from the outgoing flux. */
static int transform_wall_nodes(const oracle_params* p, double* f) {
    const int V = p->V, Nx = p->Nx, Ny = p->Ny;
    const double h = p->dt / (2.0 * p->tau);
    double* phi = malloc(sizeof(double) * V);
    int* unk = malloc(sizeof(int) * V);
    if (!phi || !unk) { free(phi); free(unk); return -1; }
    for (int y = 0; y < Ny; ++y)
        for (int x = 0; x < Nx; ++x) {
            int any = 0;
            for (int a = 0; a < V; ++a) {
                const int ys = y - p->ey[a];
                unk[a] = ys < 0 || ys >= Ny;
                if (unk[a]) { phi[a] = f[at(p, a, x, y)]; any = 1; }
            }
            if (!any) continue;
            for (int it = 0; it < 100; ++it) {
                double rho = 0.0, mx = 0.0, my = 0.0;
                for (int a = 0; a < V; ++a) {
                    const double fa = f[at(p, a, x, y)];
                    rho += fa;
                    mx += fa * p->c * p->ex[a];
                    my += fa * p->c * p->ey[a];
                }
                const double ux = (mx + 0.5 * p->dt * rho * p->gx) / rho;
                const double uy = (my + 0.5 * p->dt * rho * p->gy) / rho;
                const double uu = ux * ux + uy * uy;
                double change = 0.0;
                for (int a = 0; a < V; ++a) {
                    if (!unk[a]) continue;
                    const double s = ux * p->c * p->ex[a] + uy * p->c * p->ey[a];
                    const double f0 = rho * p->w[a] * f0_over_rho_w(p->N, s, uu);
                    const double v = (1.0 + h) * phi[a] - h * f0;
                    const double d = fabs(v - f[at(p, a, x, y)]);
                    if (d > change) change = d;
                    f[at(p, a, x, y)] = v;
                }
                if (change < 1e-16) break;
            }
        }
    free(phi);
    free(unk);
    return 0;
}

/* Steps (5) and (6): fbar(t+dt) from the post-collision field fstar. */
int oracle_stream(const oracle_params* p, const double* fstar, double* f) {
    const int V = p->V, Nx = p->Nx, Ny = p->Ny;

    /* Mass flux through each wall per column, Eq. nm.15 numerator:
     * sum over outgoing populations (e_y < 0 at the bottom wall y = 0,
     * e_y > 0 at the top wall y = Ny) of the rows that cross the wall.
     * The population leaving from (xs, j) is credited to column
     * (xs + e_x) mod Nx. */
    double* out_bot = calloc((size_t)2 * Nx, sizeof(double));
    if (!out_bot) return -1;
    double* out_top = out_bot + Nx;
    for (int a = 0; a < V; ++a) {
        int ey = p->ey[a];
        for (int xs = 0; xs < Nx; ++xs) {
            int xl = wrap(xs + p->ex[a], Nx);
            if (ey < 0)
                for (int j = 0; j < -ey; ++j) out_bot[xl] += fstar[at(p, a, xs, j)];
            if (ey > 0)
                for (int j = Ny - ey; j < Ny; ++j) out_top[xl] += fstar[at(p, a, xs, j)];
        }
    }
    /* Eq. nm.15 denominator with f0(rho_w, u = 0) = rho_w w_a: each incoming
     * population a is emitted into |e_y| rows, so the emitted mass per unit
     * Psi rho_w is sum_{incoming} |e_ay| w_a. */
    double den_bot = 0.0, den_top = 0.0;
    for (int a = 0; a < V; ++a) {
        if (p->ey[a] > 0) den_bot += p->ey[a] * p->w[a];
        if (p->ey[a] < 0) den_top += -p->ey[a] * p->w[a];
    }

#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < V; ++a)
        for (int y = 0; y < Ny; ++y)
            for (int x = 0; x < Nx; ++x) {
                int ys = y - p->ey[a];
                double v;
                if (ys < 0)
                    v = out_bot[x] / den_bot * p->w[a];      /* Eq. nm.14 */
                else if (ys >= Ny)
                    v = out_top[x] / den_top * p->w[a];
                else
                    v = fstar[at(p, a, wrap(x - p->ex[a], Nx), ys)];
                f[at(p, a, x, y)] = v;
            }
    free(out_bot);
    if (p->wall_mode == 1) return transform_wall_nodes(p, f);
    return 0;
}

int oracle_run(const oracle_params* p, double* f, double* work, long nsteps) {
    for (long n = 0; n < nsteps; ++n) {
        if (oracle_collide(p, f, work)) return -1;
        if (oracle_stream(p, work, f)) return -1;
    }
    return 0;
}

void oracle_moments(const oracle_params* p, const double* f, double* rho,
                    double* ux, double* uy) {
    for (int y = 0; y < p->Ny; ++y)
        for (int x = 0; x < p->Nx; ++x) {
            double r = 0.0, m0 = 0.0, m1 = 0.0;
            for (int a = 0; a < p->V; ++a) {
                double fa = f[at(p, a, x, y)];
                r += fa;
                m0 += fa * p->c * p->ex[a];
                m1 += fa * p->c * p->ey[a];
            }
            long i = (long)y * p->Nx + x;
            rho[i] = r;
            ux[i] = (m0 + 0.5 * p->dt * r * p->gx) / r;   /* Eq. nm.10 */
            uy[i] = (m1 + 0.5 * p->dt * r * p->gy) / r;
        }
}

/* Threads of the OpenMP build (the CPU-baseline timing); returns the count
 * in use, 1 in the serial build. */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(int n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}
#else
int oracle_threads(int n) {
    (void)n;
    return 1;
}
#endif

/* Single-node helpers exposed for the pins: equilibrium and force terms. */
void oracle_equilibrium(const oracle_params* p, double rho, double ux, double uy,
                        double* f0) {
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < p->V; ++a) {
        double s = ux * p->c * p->ex[a] + uy * p->c * p->ey[a];
        f0[a] = rho * p->w[a] * f0_over_rho_w(p->N, s, uu);
    }
}

void oracle_force(const oracle_params* p, double rho, double ux, double uy,
                  const double* Pi4, double* F) {
    const double u[2] = {ux, uy}, g[2] = {p->gx, p->gy};
    const double Pi[2][2] = {{Pi4[0], Pi4[1]}, {Pi4[2], Pi4[3]}};
    for (int a = 0; a < p->V; ++a) {
        double xi[2] = {p->c * p->ex[a], p->c * p->ey[a]};
        F[a] = force_term(p->N, p->force_a3, rho, u, g, Pi, xi, p->w[a]);
    }
}
