// Internal declarations shared by the host API (lbm_api.cu) and the kernel
// translation units (k_fp64.cu, k_fp32.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lbm.h"

namespace lbm {

constexpr int kMaxPairs = LBM_MAX_V / 2;
constexpr int kBlock = 128;          // threads per block of the step kernels

// Resident blocks per SM requested from the compiler for a register-resident
// kernel with V populations of `bytes` each: the populations plus ~30
// registers of per-node state, rounded to the allocation granularity of 8.
// More resident warps keep more loads in flight, which this HBM-bound step
// needs; the budget leaves the compiler room to avoid spills.
constexpr int min_blocks_for(int V, int bytes) {
    const int regs = ((V * bytes / 4 + (bytes == 4 ? 30 : 60)) + 7) / 8 * 8;
    const int blocks = 65536 / (regs * kBlock);
    return blocks < 1 ? 1 : (blocks > 16 ? 16 : blocks);
}
constexpr int kReduceBlocks = 304;   // 2 x 152 SMs for the partial sums
constexpr int kReduceThreads = 256;

// Per-solve constants, passed by value to every kernel (__grid_constant__).
// Planes are in the solver's internal order: R rest planes (R = 0 or 1),
// then the P "positive" members of the +-e pairs, then their P negatives in
// the same order, so plane R + P + p holds -e of plane R + p.
template <typename C>
struct KParams {
    int Nx, Ny, ncell;           // ncell = Nx * Ny
    int R, P, V;
    int maxey;                   // max |e_y|: rows within maxey of a wall
    int maxex;                   // max |e_x|
    int set_id;                  // compiled velocity set (dvm_sets.h), -1: generic
    int force;                   // 1 if g != 0
    int strips;                  // wall blocks as 32-column x 4-row strips: Nx / 32, or 0
    int emit;                    // 1: write fp64 rho, u of this step; 2: add them
    unsigned int seed;           // step counter: stochastic rounding of 16-bit stores
    long long plane;             // elements per plane = ncell
    int ex[LBM_MAX_V], ey[LBM_MAX_V];
    int sx[LBM_MAX_V];           // e_x mod Nx, in [0, Nx)
    int off[LBM_MAX_V];          // e_y Nx + e_x: pull offset of an interior node
    int dx[LBM_MAX_V];           // e_x - sx: offset correction when x - e_x wraps
    // per launch: plane base pointers of the source lattice shifted by the
    // interior pull offset (srcf[a] = src + a plane - off[a]) and of the
    // destination lattice (dstp[a] = dst + a plane)
    const void* srcf[LBM_MAX_V];
    void* dstp[LBM_MAX_V];
    double w[LBM_MAX_V];         // weights (fp64) for the initial state
    C cw[LBM_MAX_V];             // weights in the compute type, for the wall fill
    // 16-bit storage only: stored h_a = d_a / (w_a S), S a per-solve power of 2
    C sw[LBM_MAX_V];             // w_a S      (load:  d = h * sw)
    C isw[LBM_MAX_V];            // 1/(w_a S)  (store: h = d * isw)
    // 16-bit storage, compiled velocity sets: the kernels keep h itself in
    // registers; the moment sums of d = w S h weigh h with these (pair p):
    C hw[kMaxPairs], hwx[kMaxPairs], hwy[kMaxPairs];        // w S, w S e_x, w S e_y
    C hwxx[kMaxPairs], hwxy[kMaxPairs], hwyy[kMaxPairs];    // w S e_x^2, w S e_x e_y, w S e_y^2
    C hw_rest;                   // w_rest S
    C fill_h;                    // 1/S: the wall fill dPsi w_a in units of w_a S
    C om_s;                      // omega / S: relaxation target in units of w_a S
    double inv_den;              // 1 / sum_{e_y > 0} e_y w  (= same for e_y < 0)
    // per pair p, positive member e = (ex, ey):
    C pex[kMaxPairs], pey[kMaxPairs];
    C pexx[kMaxPairs], pexy2[kMaxPairs], peyy[kMaxPairs];   // ex^2, 2 ex ey, ey^2
    C pge[kMaxPairs];            // c g.e
    C pomw[kMaxPairs];           // omega w_p
    C omw_rest;                  // omega w_rest
    // scalars
    C c, c2, tau, dt, hdt, omega, one_m_omega, gx, gy;
    C two_tau, inv_2tau_dt, half_tau;
    // products of constants (formed on the host in C, as the device would):
    // hdt gx, hdt gy, two_tau gx, two_tau gy, two_tau c2, half_tau c2, tau c, c gx
    C hdt_gx, hdt_gy, tgx, tgy, ttc2, htc2, tc, cg;
};

// Device buffers of one solver.
struct DevBufs {
    void* f[2];                  // population lattices (ping-pong)
    double* rho;                 // fp64 moments of the latest state
    double* ux;
    double* uy;
    double* prev_ux;             // u_x one step earlier (convergence test); init staging
    double* partial;             // 2 * kReduceBlocks reduction scratch
    double* results;             // 8 doubles: mean_ux, max_du, u_s, mdot, ...
    unsigned int* status;        // bit 0: non-finite / non-positive density
};

// Kernel launchers, one set per precision (k_fp64.cu, k_fp32.cu).
// Return cudaSuccess or the launch error.
cudaError_t launch_step_fp64(const KParams<double>& k, int N, const void* src,
                             void* dst, const DevBufs& b, cudaStream_t st);
cudaError_t launch_init_fp64(const KParams<double>& k, int N, const double* rho0,
                             void* dst, const DevBufs& b, cudaStream_t st);
cudaError_t launch_step_fp32(const KParams<float>& k, int N, const void* src,
                             void* dst, const DevBufs& b, cudaStream_t st);
cudaError_t launch_init_fp32(const KParams<float>& k, int N, const double* rho0,
                             void* dst, const DevBufs& b, cudaStream_t st);
// 16-bit storage (fp32 arithmetic): bf16 = false -> IEEE half, true -> bfloat16
cudaError_t launch_step_fp16(const KParams<float>& k, int N, bool bf16, const void* src,
                             void* dst, const DevBufs& b, cudaStream_t st);
cudaError_t launch_init_fp16(const KParams<float>& k, int N, bool bf16, const double* rho0,
                             void* dst, const DevBufs& b, cudaStream_t st);
// max over the stored state of |h| (16-bit storage), into *out (device)
cudaError_t launch_absmax_fp16(const void* f, long long n, bool bf16, float* out,
                               cudaStream_t st);
// multiply every stored value by `factor` (a power of 2)
cudaError_t launch_rescale_fp16(void* f, long long n, bool bf16, float factor,
                                cudaStream_t st);

// Tiny fp64 / fp32 channels: lanes per node of the warp step (k_step_warp) for P pairs,
// 0 when the channel is large enough for one node per thread (or P > 32).
inline int warp_lanes(int P) { return P <= 8 ? 8 : (P <= 16 ? 16 : (P <= 32 ? 32 : 0)); }
inline int warp_path_lanes(int P, long long ncell) {
    const int LP = warp_lanes(P);
    return (LP && ncell * LP <= 152ll * 32 * 8) ? LP : 0;
}

// Resident chunks of a tiny fp64 or fp32 channel on one thread-block cluster
// (k_cluster.cu): CTAs of at most kClusterThreads threads, shared memory padded
// to kClusterSmemPad (more than half an SM's) so that no two share an SM.
constexpr int kClusterThreads = 256;
constexpr int kClusterSmemPad = 116 * 1024;
constexpr long kClusterMaxK = 4096;           // steps per launch in lbm_step
struct ClusterPlan {
    int ctas = 0, rows = 0, threads = 0, N = 0, LP = 0;
    int nb = 0, nt = 0;                       // terms of the bottom / top wall sums
    size_t smem = 0;
};
// 1 and the plan if the channel can run resident, else 0 (pl.ctas = 0).
int plan_cluster(const KParams<double>& k, int N, int LP, ClusterPlan& pl);
int plan_cluster(const KParams<float>& k, int N, int LP, ClusterPlan& pl);
// K steps from fin to fout (see k_chunk_cluster).
cudaError_t launch_chunk_cluster(const KParams<double>& k, const ClusterPlan& pl, const void* fin,
                                 void* fout, const DevBufs& b, int K, bool emit_prev,
                                 cudaStream_t st);
cudaError_t launch_chunk_cluster(const KParams<float>& k, const ClusterPlan& pl, const void* fin,
                                 void* fout, const DevBufs& b, int K, bool emit_prev,
                                 cudaStream_t st);

// Validated, canonicalised description of one channel solve (shared by the
// single-solve API and the engine).
struct SolveSpec {
    int precision = LBM_FP64;
    int N = 3, Nx = 1, Ny = 1, V = 0, R = 0, P = 0, maxey = 0, maxex = 0, set_id = -1;
    double c = 1, Kn = 0, tau = 0, dt = 0, g = 0, den = 0;
    double scale = 1.0 / 64.0;   // S of the 16-bit storage (power of 2)
    size_t elem = 8;
    std::vector<int> perm;       // internal plane -> caller velocity index
    std::vector<int> ex, ey;     // internal order
    std::vector<double> w;
};

// Validate the arguments of lbm_create and fill `s` (LBM_OK or an error code).
int prepare_spec(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn, double force,
                 int precision, SolveSpec& s);
template <typename C>
void fill_params(const SolveSpec& s, KParams<C>& k);
size_t elem_bytes(int precision);

}  // namespace lbm
