/* Sanitizer run of the oracle time step (test infrastructure).
 * Reads "V c N Nx Ny Kn g steps wall_mode force_a3" then V lines "ex ey w"
 * from stdin, runs the steps from rho = 1 and prints the relative change of the
 * total mass and the centre velocity. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm_oracle.h"

int main(void) {
    int V, N, Nx, Ny, wall_mode, force_a3;
    long steps;
    double c, Kn, g;
    if (scanf("%d %lf %d %d %d %lf %lf %ld %d %d", &V, &c, &N, &Nx, &Ny, &Kn, &g, &steps,
              &wall_mode, &force_a3) != 10)
        return 2;
    int* ex = malloc(sizeof(int) * V);
    int* ey = malloc(sizeof(int) * V);
    double* w = malloc(sizeof(double) * V);
    for (int a = 0; a < V; ++a)
        if (scanf("%d %d %lf", &ex[a], &ey[a], &w[a]) != 3) return 2;
    oracle_params p = {V, Nx, Ny, N, ex, ey, w, c, sqrt(2.0 / M_PI) * Kn, 1.0 / (Ny * c), g, 0.0,
                       wall_mode, force_a3};
    const long n = (long)V * Nx * Ny;
    double* f = malloc(sizeof(double) * n);
    double* work = malloc(sizeof(double) * n);
    for (int a = 0; a < V; ++a)
        for (long i = 0; i < (long)Nx * Ny; ++i) f[(long)a * Nx * Ny + i] = w[a];
    double m0 = 0.0, m1 = 0.0;
    for (long i = 0; i < n; ++i) m0 += f[i];
    if (oracle_run(&p, f, work, steps)) return 3;
    for (long i = 0; i < n; ++i) m1 += f[i];
    double* rho = malloc(sizeof(double) * Nx * Ny);
    double* ux = malloc(sizeof(double) * Nx * Ny);
    double* uy = malloc(sizeof(double) * Nx * Ny);
    oracle_moments(&p, f, rho, ux, uy);
    printf("%.3e %.6e\n", fabs(m1 / m0 - 1.0), ux[(Ny / 2) * Nx]);
    free(ex); free(ey); free(w); free(f); free(work); free(rho); free(ux); free(uy);
    return 0;
}
