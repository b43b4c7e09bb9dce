/*
 * lbm.h - C ABI of the GB300 high-order lattice Boltzmann channel solver.
 *
 * One solver = one force-driven plane channel (Feuchter & Schleifenbaum,
 * "High-order lattice Boltzmann models for wall-bounded flows at finite
 * Knudsen numbers", Sect. V and VI): Nx nodes along the periodic stream
 * direction x, Ny nodes between two diffuse Maxwell walls at rest, a
 * constant body acceleration g along x.  Every time step runs on the GPU:
 * pull streaming, the diffuse-wall flux balance, moments, the order-N Hermite
 * equilibrium, the body-force term and the trapezoidal BGK relaxation, fused
 * in one kernel (Eq. nm.3, nm.4, nm.8, nm.10, nm.14, nm.15).
 *
 * Units (Sect. II, V): lengths in l0 = channel width, velocities in
 * c0 = sqrt(R theta0), times in l0/c0.  Node j sits at y = (j + 1/2) dx with
 * dx = 1/Ny, half a spacing from each wall (Sect. V).  dt = dx / c, so one
 * step moves population a by its integer velocity e_a.  tau = sqrt(2/pi) Kn
 * (Eq. nm.13).
 *
 * Conventions for every call:
 *  - Every function returns LBM_OK (0) or a negative LBM_E* code; nothing
 *    throws across the ABI and no call traps the device.
 *  - "host" buffers are caller-owned CPU memory, "device" buffers are
 *    caller-owned GPU memory on the solver's device.
 *  - Calls are asynchronous on the solver's CUDA stream, except those that
 *    return host values (lbm_moments, lbm_mass_flow, lbm_slip_velocity,
 *    lbm_run_to_steady, lbm_status, lbm_get_state, lbm_populations), which
 *    synchronise that stream before returning.
 *  - A solver is not thread-safe: one host thread drives it at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,      /* invalid argument (sizes, Kn, weights, pointers)   */
    LBM_EDEGREE = -2,     /* quadrature order too low for the Hermite order    */
    LBM_ENOMEM = -3,      /* device allocation failed / workspace too small    */
    LBM_ECUDA = -4,       /* a CUDA runtime call failed                        */
    LBM_ENONFINITE = -5,  /* a non-finite or non-positive density appeared     */
    LBM_ETIMEOUT = -6,    /* a bounded device wait gave up                     */
    LBM_ENOTCONV = -7,    /* lbm_run_to_steady reached max_steps               */
    LBM_ENOTSUP = -8      /* valid but not supported by this build             */
};

/* Storage precision of the populations.  Every precision stores the
 * deviation d_a = fbar_a - w_a from the rest state at rho0 = 1.
 *   LBM_FP64: d in fp64, fp64 arithmetic;
 *   LBM_FP32: d in fp32, fp32 arithmetic;
 *   LBM_FP16, LBM_BF16: h_a = d_a / (w_a S) in IEEE half / bfloat16, fp32
 *     arithmetic; S is a per-solve power of 2 (initially 2^-6) that
 *     lbm_run_to_steady refreshes at every test so that max |h| is in (1/2, 1].
 * The wall flux balance, the moments handed to the host and every reduction
 * are fp64 in all precisions. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_BF16 = 3 };

/* A two-dimensional discrete velocity model (Sect. II.A): velocities
 * xi_a = c e_a with integer e_a, weights w_a.  The set must be closed under
 * e -> -e with equal weights (all DVMs of the paper are), sum w_a = 1 to
 * 1e-12, V <= LBM_MAX_V.  Caller-owned; copied by lbm_create. */
#define LBM_MAX_V 128
typedef struct {
    int D;               /* must be 2                                       */
    int V;               /* number of velocities                            */
    const int* e;        /* V*2 ints, row-major (e_x, e_y), y = wall normal */
    const double* w;     /* V weights                                       */
    double c;            /* lattice speed                                   */
} lbm_dvm;

typedef struct lbm_solver lbm_solver;   /* opaque */

/* ---- DVM utilities (host only, no GPU needed) --------------------------- */

/* Expand printed symmetry groups into velocities (Eq. wdach): each
 * representative reps[g*D .. g*D+D-1] (D = 2 or 3) generates the orbit under
 * all component permutations and sign flips; every member gets weight wg[g].
 * vg[g], if not NULL, is the group size the caller expects (checked).
 * Outputs up to cap velocities into e_out (V*D ints) and w_out.
 * Errors: LBM_EINVAL on a size mismatch or cap too small. */
int lbm_dvm_expand(int D, int G, const int* reps, const int* vg, const double* wg,
                   int cap, int* e_out, double* w_out, int* V_out);

/* (x, z) marginal of a 3D set e3 (V3*3 ints, (x, y, z)): weights of
 * velocities sharing (e_x, e_z) are summed.  Exact for flows uniform along y,
 * the paper's channel (Sect. VI).  Output order: sorted by (e_x, e_z). */
int lbm_dvm_marginal_xz(int V3, const int* e3, const double* w3, int cap,
                        int* e2_out, double* w2_out, int* V2_out);

/* Quadrature order Q of a 2D DVM (Eq. orth): the largest degree up to 16 for
 * which every moment sum_a w_a xi_ax^i xi_ay^j, i + j <= Q, equals the
 * Gaussian moment (i-1)!!(j-1)!! (relative tolerance 1e-9). */
int lbm_dvm_quadrature_order(const lbm_dvm* dvm, int* Q_out);

/* ---- DVM generator (host only, no GPU needed) ---------------------------- */
/* Velocities: e[V*D] ints, row-major, D = 2 (x, z) or 3 (x, y, z), the last
 * component the wall normal; multiples of the lattice speed c.  The stencil
 * must be closed under the lattice reflections (component permutations and
 * sign flips), else LBM_EINVAL.  1 <= Q <= 16. */

/* Weights of a stencil (Sect. III): the normalised (sum w = 1) null vector
 * of K(S) (Eq. defQua, defK), one weight per symmetry group (Eq. wdach).
 * *nullity_out = dim ker K (Eq. dimker): 1 for a DVM of order Q at this c
 * (weights in w_out[V]); 0 when K(S) is regular (c is not a c*); > 1 when
 * the weights are not unique (see lbm_dvm_augment).  w_out is NaN unless
 * the nullity is 1.  Null directions: singular values of the per-group
 * orthogonality conditions below 1e-9 of the largest. */
int lbm_dvm_solve_weights(int D, int V, const int* e, double c, int Q, double* w_out,
                          int* nullity_out);

/* Lattice speed c* in [c_lo, c_hi] at which the stencil is a minimal DVM
 * of order Q (dim ker K = 1) with positive weights (Eq. dimker): the
 * smallest such c*, located to rounding (400-point scan, golden-section
 * refinement).  LBM_ENOTCONV if there is none in the interval. */
int lbm_dvm_find_c(int D, int V, const int* e, int Q, double c_lo, double c_hi,
                   double* c_out);

/* The L non-trivial equilibrium wall moments (m_x, m_y, m_z) of Eq. nontriv
 * in the paper's order (increasing n, decreasing m_z, decreasing m_x;
 * m_y = 0 in 2D), 3 ints each into m_out (cap moments; NULL with cap 0
 * returns only *L_out). */
int lbm_dvm_nontrivial_moments(int D, int Q, int cap, int* m_out, int* L_out);

/* Wall-augmented weights (Sect. IV): w = x_j w^(j) over a basis of the null
 * space of K(S) (Eq. 9.13), x from A x = b (Eq. wallEq, defA) for the nk
 * selected non-trivial wall moments k[] (indices into
 * lbm_dvm_nontrivial_moments), b their exact values (Eq. Wscalar), together
 * with sum w = 1; least squares when overdetermined, minimum norm when
 * underdetermined.  w_out[V]; *residual_out (may be NULL) = |A x - b|.
 * LBM_EDEGREE if K(S) is regular at c. */
int lbm_dvm_augment(int D, int V, const int* e, double c, int Q, int nk, const int* k,
                    double* w_out, double* residual_out);

/* ---- solver lifetime ---------------------------------------------------- */

/* Device bytes lbm_create_in needs for this problem (both population
 * lattices, fp64 moment fields, reduction scratch). */
int lbm_workspace_bytes(const lbm_dvm* dvm, int Nx, int Ny, int precision,
                        size_t* bytes);

/* Create a solver that allocates its own device memory with cudaMalloc on the
 * current device.
 *   order: Hermite order N of the equilibrium, 2 <= N <= 4 and Q >= 2N - 1
 *          (Sect. III: N = (Q-1)/2 is optimal, (Q+1)/2 still admissible);
 *          otherwise LBM_EDEGREE.  Q must also be >= 5.
 *   Nx >= 1 (periodic), Ny >= max |e_y| (walls), Kn > 0, force = g_x
 *   (0 allowed: then lbm_mass_flow returns mdot = NaN).
 *   precision: LBM_FP64, LBM_FP32, LBM_FP16 or LBM_BF16.
 *   stream: a cudaStream_t, or NULL for the legacy default stream.
 * The state is undefined until lbm_init. */
int lbm_create(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn,
               double force, int precision, void* stream, lbm_solver** out);

/* As lbm_create, but uses caller-owned device memory `workspace` of `bytes`
 * (>= lbm_workspace_bytes; 256-byte aligned) instead of allocating; the
 * workspace must outlive the solver.  LBM_ENOMEM if bytes is too small. */
int lbm_create_in(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn,
                  double force, int precision, void* stream, void* workspace,
                  size_t bytes, lbm_solver** out);

/* Release the solver (and its memory, if lbm_create allocated it). */
void lbm_destroy(lbm_solver* s);

const char* lbm_strerror(int code);

/* ---- state ------------------------------------------------------------- */

/* Initial state fbar_a = rho(x, y) w_a (fluid at rest).  rho_host: Ny*Nx
 * doubles, row-major [y][x], copied host->device; NULL means rho = 1.
 * Resets the step counter and the status word. */
int lbm_init(lbm_solver* s, const double* rho_host);

/* As lbm_init with rho already in device memory (Ny*Nx doubles). */
int lbm_init_device(lbm_solver* s, const double* rho_device);

/* Advance nsteps >= 0 time steps (Eq. nm.8 + streaming + walls), one fused
 * kernel launch per step on the solver's stream, or, for a resident channel
 * (lbm_set_resident), up to 4096 steps per launch.  Asynchronous. */
int lbm_step(lbm_solver* s, long nsteps);

/* Resident chunks for tiny fp64 and fp32 channels (no counterpart in the
 * paper, which does not discuss execution).  A channel whose step runs on
 * several lanes per node (at most 152*32*8 node-lanes) and whose rows fit one
 * thread-block cluster (at most 16 CTAs of at most 8 warps, both lattices in
 * their shared memory) runs many steps per launch, the cluster's barrier
 * between steps, instead of one launch per step; lbm_step and
 * lbm_run_to_steady then use it.  The result is bitwise that of the per-step
 * launches.  enable: 1 (the default at lbm_create) or 0; anything else ->
 * LBM_EINVAL.  16-bit storage and larger channels ignore the setting. */
int lbm_set_resident(lbm_solver* s, int enable);

/* *ctas = CTAs of the cluster that runs this solver's resident chunks, 0 when
 * it steps by single launches (not eligible, not placeable on this device, or
 * disabled).  NULL pointer -> LBM_EINVAL. */
int lbm_resident_ctas(lbm_solver* s, int* ctas);

/* Time-averaged moments.  The paper's scheme is deterministic; 16-bit
 * storage with stochastically rounded stores (LBM_FP16, LBM_BF16) is not: its
 * state settles into a statistical steady state whose snapshots scatter by
 * the rounding noise (~1e-3 of the flow in u_s at the walls), while time
 * averages converge to the steady state of the scheme.  lbm_average advances
 * nsteps steps and samples the fp64 moments rho, u_x, u_y of every `every`-th
 * of them (floor(nsteps / every) samples); afterwards the moment fields hold
 * the sample means, so lbm_moments, lbm_mass_flow, lbm_slip_velocity and
 * lbm_knudsen_layer report time averages (mass flow and slip velocity of the
 * averaged field, Eq. pf.1 and defSlip) until the next step.  The state
 * itself is the last step's.  Any precision; one launch per step.
 * Requires nsteps >= every >= 1, else LBM_EINVAL.  Asynchronous. */
int lbm_average(lbm_solver* s, long nsteps, long every);

/* Step until max over nodes of |u_x(t) - u_x(t - dt)| < tol, tested every
 * check_every (>= 2) steps, or until max_steps in total.  Returns LBM_OK when
 * converged, LBM_ENOTCONV otherwise; *steps_done and *last_du (either may be
 * NULL) report the total steps and the last tested change. */
int lbm_run_to_steady(lbm_solver* s, double tol, long max_steps,
                      long check_every, long* steps_done, double* last_du);

/* Moments of the current state (Eq. nm.10): rho, u_x, u_y in units of rho0
 * and c0, each Ny*Nx doubles [y][x] (host).  Any pointer may be NULL. */
int lbm_moments(lbm_solver* s, double* rho, double* ux, double* uy);

/* Normalised mass flow (Eq. pf.1) mdot = 2 tau <u_x> / (g Kn), <u_x> the
 * mean over all nodes (midpoint rule).  Either pointer may be NULL. */
int lbm_mass_flow(lbm_solver* s, double* mdot, double* mean_ux);

/* Slip velocity u_s = u(wall)/u(centre) (Eq. defSlip).  u(wall): quadratic
 * extrapolation (15 u_0 - 10 u_1 + 3 u_2)/8 from the three nodes nearest to
 * each wall, averaged over both walls and all x; u(centre): the centre node
 * for odd Ny, the four-point midpoint interpolation
 * (9(u_{m-1} + u_m) - (u_{m-2} + u_{m+1}))/16, m = Ny/2, for even Ny.
 * Needs Ny >= 4. */
int lbm_slip_velocity(lbm_solver* s, double* us);

/* Knudsen-layer diagnostic (Eq. uNS, uNEQ): u_neq(y) = u(y) - u_NS(y) for the
 * x-averaged velocity u(y) of the current state, u_NS the parabola through the
 * centre value u(0) (as in lbm_slip_velocity) with the same mass flow:
 * u_NS(y) = u(0) (1 - 3 (1 - <u>/u(0)) (2 z)^2), z = (y + 1/2)/Ny - 1/2, <u>
 * the mean over all nodes.  uneq: Ny doubles (host).  Needs Ny >= 4.  Uses the
 * solver's convergence-reference field as scratch. */
int lbm_knudsen_layer(lbm_solver* s, double* uneq);

/* Device status word: LBM_OK, or LBM_ENONFINITE once any step met a
 * non-finite or non-positive density.  Synchronises the stream. */
int lbm_status(lbm_solver* s);

/* Steps taken since lbm_init. */
int lbm_steps_done(lbm_solver* s, long* steps);

/* Post-collision populations fbar*_a(x, y) of the last step (the state the
 * next streaming step reads), as fp64, V*Ny*Nx doubles, planes in the
 * caller's velocity order [a][y][x] (host). */
int lbm_populations(lbm_solver* s, double* f_host);

/* Checkpoint / resume: an opaque byte image of the state (populations in
 * storage precision, moment fields, step counter).  lbm_state_bytes gives the
 * size; restoring into a solver created with the same arguments continues
 * bit-identically. */
int lbm_state_bytes(lbm_solver* s, size_t* bytes);
int lbm_get_state(lbm_solver* s, void* host, size_t bytes);
int lbm_set_state(lbm_solver* s, const void* host, size_t bytes);

/* ---- multi-solve engine (batched channels, continuous batching) -------- */

/* An engine advances many independent channel solves together: each time
 * step is one persistent kernel launch per velocity set present, whose blocks
 * take 128-node tiles of any resident solve from a shared work counter, so
 * solves of uneven sizes share the GPU without one launch per solve.  A chunk
 * of K steps (default 100) plus the per-solve fp64 reductions is captured once
 * in a CUDA graph and replayed.  Solves can be added and removed between
 * chunks; their populations stay resident in the engine's arena, and a solve
 * is admitted only if its footprint (lbm_engine_solve_bytes) fits.
 * Supported: the velocity sets with compiled kernels (the paper's D2V16,
 * D2V32, D2V33 and the (x, z) marginals of D3V107, D3V96, D3V112;
 * LBM_ENOTSUP otherwise), storage LBM_FP64 (fp64 arithmetic), LBM_FP32,
 * LBM_FP16 or LBM_BF16 (fp32 arithmetic; the 16-bit scale S stays 2^-6 in the
 * engine).  Each solve's arithmetic is the one of lbm_step's compiled-set
 * kernel, so a solve's results do not depend on which other solves share the
 * engine.  Not thread-safe. */
typedef struct lbm_engine lbm_engine;

/* Device bytes one solve occupies in an engine arena. */
int lbm_engine_solve_bytes(const lbm_dvm* dvm, int Nx, int Ny, int precision,
                           size_t* bytes);

/* arena: caller-owned device memory of arena_bytes (256-byte aligned), or
 * NULL to cudaMalloc arena_bytes.  The engine's control data (slot records,
 * tile lists) is carved from the start of the arena.  max_solves: slots.
 * stream: a cudaStream_t other than the legacy default stream, or NULL to
 * let the engine create one (graph capture needs a non-default stream). */
int lbm_engine_create(int precision, int max_solves, void* arena, size_t arena_bytes,
                      void* stream, lbm_engine** out);
void lbm_engine_destroy(lbm_engine* e);

/* Admit a solve (arguments as lbm_create; rho_host as lbm_init) and
 * initialise it.  *slot receives its slot index.  LBM_ENOMEM when no slot is
 * free or its footprint does not fit in the arena (the caller may retry after
 * a removal).  Asynchronous on the engine's stream (rho_host is copied before
 * the call returns); errors of the queued work surface at the next
 * lbm_engine_run. */
int lbm_engine_add(lbm_engine* e, const lbm_dvm* dvm, int order, int Nx, int Ny,
                   double Kn, double force, const double* rho_host, int* slot);

/* Release a slot and its arena memory.  Stream-ordered: work already queued
 * for the slot completes before a later solve can use its memory. */
int lbm_engine_remove(lbm_engine* e, int slot);

/* Steps per chunk, even, 2..1000 (default 100). */
int lbm_engine_set_chunk(lbm_engine* e, int steps);

/* Resident chunks on (1, the default) or off (0).  When on, solves whose
 * populations fit in one block's shared memory (V Nx (Ny + 2 max|e_y|)
 * elements, at most 4096 nodes) are packed into bundles, and each bundle
 * advances a whole chunk inside shared memory (one launch per chunk and
 * velocity set), reading and writing device memory once per chunk.  The
 * other solves take one tiled launch per step.  Both give bitwise the same
 * results.  Takes effect at the next lbm_engine_run or
 * lbm_engine_autotune.  LBM_EINVAL unless enable is 0 or 1. */
int lbm_engine_set_resident(lbm_engine* e, int enable);

/* How many solves take each path at the next chunk: per-step tiles and
 * resident (shared-memory) bundles.  Either pointer may be NULL.  Applies
 * pending admissions and removals (as lbm_engine_run would). */
int lbm_engine_paths(lbm_engine* e, int* tiled, int* resident);

/* Advance every resident solve by chunks * K steps, then copy the per-slot
 * results to `results` (host, 4 * max_solves doubles, may be NULL):
 * results[4 s + 0] = max |u_x(t) - u_x(t - dt)| over the last step,
 * [4 s + 1] = mdot (Eq. pf.1), [4 s + 2] = u_s (Eq. defSlip), [4 s + 3] =
 * <u_x>; entries of free slots are stale.  Synchronises. */
int lbm_engine_run(lbm_engine* e, int chunks, double* results);

/* Asynchronous form of lbm_engine_run, so that the host can prepare the next
 * chunk while the GPU runs this one.  lbm_engine_launch queues chunks * K
 * steps (with the solves resident at the call) and an in-stream copy of the
 * per-slot results after them into pinned host memory, and returns at once;
 * lbm_engine_wait waits for the oldest outstanding launch and copies its
 * results (layout as lbm_engine_run) to `results` (may be NULL).  At most two
 * launches may be outstanding (LBM_EINVAL otherwise, and for a wait with none
 * outstanding).  Adding or removing solves between a launch and its wait is
 * allowed and stream-ordered: a removed solve is still advanced by the
 * launches queued before its removal, and results of a slot refer to the
 * solve it held when that launch was queued.  lbm_engine_run and
 * lbm_engine_autotune return LBM_EINVAL while launches are outstanding. */
int lbm_engine_launch(lbm_engine* e, int chunks);
int lbm_engine_wait(lbm_engine* e, double* results);

/* Time candidate schedules of the tiled kernel on the resident solves and
 * keep the fastest.  Each velocity-set group (set and Hermite order) with
 * tiled solves has its own tile shape, cells per tile and tiles per grab.
 * The groups run together in a chunk, so every candidate is timed on the
 * whole chunk (two chunks after a warm-up chunk).  The search: the 11 tile
 * shapes (linear tiles of 128, 256 or 512 consecutive nodes; rectangles 32 or
 * 64 columns wide of 128, 256 or 512 nodes, or 128 wide of 256 or 512) for
 * all groups at once; then, group by group, its own shape and its tiles per
 * grab (1, 2, 4, 8 or 16), a change kept only when it saves more than 0.5 %;
 * last the persistent grid at 1 or 1/2 of the occupancy limit.  The schedule
 * decides which block updates a node, never the node's arithmetic: results
 * are bitwise the same under every schedule.  The timed chunks advance the
 * solves (3 chunks per candidate, counted in their step counters; 12 + 14 G
 * candidates for G tiled groups from the default schedule).
 * *best_ms_per_step (may be NULL) receives the time of one step of the best
 * candidate. */
int lbm_engine_autotune(lbm_engine* e, double* best_ms_per_step);

/* Set or read a schedule.  slot: a used slot, addressing its velocity-set
 * group, or -1 (set only) for every group.  tile_width: 0 for linear tiles
 * (consecutive nodes in row-major order), else 32, 64 or 128 columns (a
 * solve whose Nx is not a multiple of it, or whose Ny is below the tile's
 * rows, takes linear tiles); tile_cells: nodes per tile, 128, 256 or 512;
 * grab: tiles taken per atomic grab, 1..64; grid_fraction: fraction of the
 * occupancy limit used for the persistent grid, (0, 1], common to all groups.
 * LBM_EINVAL for other values, an unused slot, or while launches are
 * outstanding.  Takes effect at the next lbm_engine_run or
 * lbm_engine_launch.  Any output pointer of the getter may be NULL. */
int lbm_engine_set_schedule(lbm_engine* e, int slot, int tile_width, int tile_cells, int grab,
                            double grid_fraction);
int lbm_engine_get_schedule(const lbm_engine* e, int slot, int* tile_width, int* tile_cells,
                            int* grab, double* grid_fraction);

/* Steps done by a slot and its status (LBM_OK or LBM_ENONFINITE). */
int lbm_engine_info(lbm_engine* e, int slot, long* steps, int* status);

/* Moments of a slot's state after the last chunk (as lbm_moments). */
int lbm_engine_moments(lbm_engine* e, int slot, double* rho, double* ux, double* uy);

/* Largest contiguous free block of the arena. */
int lbm_engine_free_bytes(lbm_engine* e, size_t* largest);

/* Checkpoint of one slot: a 64-byte header (V, Nx, Ny, precision, steps),
 * the populations in storage format (V planes of Nx Ny elements, deviation
 * form as lbm_populations describes) and the four fp64 moment fields (rho,
 * u_x, u_y, previous u_x).  lbm_engine_state_bytes gives the size.
 * lbm_engine_set_state restores into a slot holding a solve of the same
 * velocity set, order, size and precision (LBM_EINVAL otherwise); fp32 solves
 * then continue bit-identically, 16-bit solves continue with the stochastic
 * rounding stream of their new slot.  Both synchronise the engine's stream. */
int lbm_engine_state_bytes(lbm_engine* e, int slot, size_t* bytes);
int lbm_engine_get_state(lbm_engine* e, int slot, void* host, size_t bytes);
int lbm_engine_set_state(lbm_engine* e, int slot, const void* host, size_t bytes);

/* ---- measurement helper -------------------------------------------------- */

/* Sustained FMA rate of the current device (no counterpart in the paper: the
 * roofline denominator of an arithmetic-bound step).  precision: LBM_FP64 or
 * LBM_FP32 (else LBM_EINVAL).  Launches a grid of 8 blocks per SM, each thread
 * running 8 independent chains a = a b + c, timed with CUDA events on
 * `stream` (a cudaStream_t or NULL) after an untimed launch; *flops_per_s is
 * the best of three, counting 2 flops per FMA.  Allocates and frees a small
 * device buffer; synchronises the stream.  Takes ~0.1-0.3 s on GB300. */
int lbm_fma_rate(int precision, void* stream, double* flops_per_s);

/* ---- observables without allocation ------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory at all: a host process whose device
 * memory is entirely owned by another runtime's pool allocator, or a loop that
 * must not call cudaMalloc because the allocation would synchronise the
 * device.  It computes the same observables as lbm_mass_flow and
 * lbm_slip_velocity, but from a velocity field the caller owns, and it
 * allocates nothing.
 *
 *   ux_device:  Ny*Nx doubles, row-major [y][x], u_x in units of c0 (device)
 *   Nx >= 1, Ny >= 4, Nx*Ny <= 16,777,216 (larger fields: LBM_EINVAL)
 *   Kn > 0, force = g_x: as in lbm_create (tau = sqrt(2/pi) Kn)
 *   out_device: 3 doubles (device), written {<u_x>, mdot, u_s}; mdot is NaN
 *               when force == 0
 *   stream:     a cudaStream_t or NULL; the call is asynchronous on it
 *
 * Its scratch is one fixed array of 4096 doubles (32 KiB) in the library's
 * device memory; every GPU that loads the library holds it until the process
 * exits.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress, with that device current), and so does the first
 * call after the device's context has changed (e.g. after cudaDeviceReset).
 * With lazy module loading (the CUDA default) that first call also loads the
 * library's kernels and the array onto the device, which takes device memory
 * and may synchronise the device: "allocates nothing" holds from the second
 * call on a device.  Make that first call before any stream capture, and
 * again after a context reset.  Every call on a device shares the array, and
 * a call overwrites every entry it reads before reading it, so nothing
 * carries over from the previous call; calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * A CUDA error already pending on the calling thread when the call starts
 * (from earlier, unrelated work) is left in place for its owner and the call
 * returns LBM_ECUDA without launching; a launch error of this call is
 * returned as LBM_ECUDA and cleared. */
int lbm_observables_noalloc(const double* ux_device, int Nx, int Ny, double Kn,
                            double force, double* out_device, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
