/* Oracle interface (test infrastructure only; never included by the library).
 * See lbm_oracle.c for the steps and the paper passages they follow. */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

typedef struct {
    int V, Nx, Ny, N;          /* velocities, channel nodes, Hermite order   */
    const int* ex;             /* V integer x components (xi = c e)          */
    const int* ey;             /* V integer y components, y = wall normal    */
    const double* w;           /* V weights                                  */
    double c;                  /* lattice speed                              */
    double tau;                /* relaxation time, units of l0/c0            */
    double dt;                 /* time step = dx / c, dx = 1/Ny              */
    double gx, gy;             /* body acceleration                          */
    int wall_mode;             /* 0: unknown fbar = Psi rho_w w_a (reading c1);
                                  1: the wall condition on f, carried to fbar
                                  through Eq. nm.7 (oracle_stream)            */
    int force_a3;              /* N = 4 only: 0: Eq. nm.4 unchanged (reading c5);
                                  1: plus the fourth-order Hermite force term
                                  with a^(3) = rho u u u                      */
} oracle_params;

/* f, work: V*Ny*Nx doubles, planes [V][Ny][Nx].  f holds fbar before the
 * collision; after oracle_run it holds fbar before the collision at t+n dt. */
int oracle_run(const oracle_params* p, double* f, double* work, long nsteps);
int oracle_collide(const oracle_params* p, const double* f, double* fstar);
int oracle_stream(const oracle_params* p, const double* fstar, double* f);
void oracle_moments(const oracle_params* p, const double* f, double* rho,
                    double* ux, double* uy);
void oracle_equilibrium(const oracle_params* p, double rho, double ux,
                        double uy, double* f0);
/* OpenMP build: set (n > 0) and return the thread count; serial build: 1. */
int oracle_threads(int n);
/* Pi4 = {Pi_xx, Pi_xy, Pi_yx, Pi_yy} */
void oracle_force(const oracle_params* p, double rho, double ux, double uy,
                  const double* Pi4, double* F);

#endif
