// Device code of the multi-solve engine: one time step of many independent
// channels in one persistent launch per compiled velocity set.
//
// Work is a list of tiles (solve slot, first node) of kBlock consecutive
// nodes of one channel.  Blocks of a fixed, SM-filling grid take `chunk`
// tiles at a time from an atomic counter, so small and large channels, wall
// tiles and interior tiles balance across the GPU.  Each tile runs the same
// arithmetic as the single-solve kernel k_step_ct (pull + walls + moments +
// relaxation), with the solve's constants read from its device record.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// Device record of one engine slot.
template <typename C>
struct EngineSolve {
    KParams<C> k;           // constants of the solve (srcf/dstp unused)
    void* f[2];             // the two population lattices
    double* rho;            // fp64 moments of the latest emitted state
    double* ux;
    double* uy;
    double* prev;           // u_x one step earlier (convergence test)
    unsigned int* status;   // bit 0: non-finite / non-positive density
    int phase;              // lattice holding the state at the start of a chunk
    int pad;
    double kn, tau, g;      // for mdot = 2 tau <u_x> / (g Kn)
};

struct EngineTile {
    int slot;
    int cell0;
};

// emit: 0 = nothing, 1 = rho, u_x, u_y into the moment fields, 2 = u_x into prev
template <class SET, int N, typename S, typename C>
__global__ void __launch_bounds__(kBlock, min_blocks_for(SET::R + 2 * SET::P + (SET::P > 20 ? 24 : 12),
                                                         sizeof(C)))
k_engine_step(const EngineSolve<C>* __restrict__ solves, const EngineTile* __restrict__ tiles,
              const int* __restrict__ ntiles_p, int* __restrict__ counter,
              const unsigned int* __restrict__ seed_p, int parity, int emit, int chunk) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P;
    __shared__ const S* sp[V];
    __shared__ S* dp[V];
    __shared__ int s_first;
    const int ntiles = *ntiles_p;
    const unsigned seed = *seed_p + unsigned(parity);
    int cur_slot = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_first = atomicAdd(counter, chunk);
        __syncthreads();
        const int first = s_first;
        if (first >= ntiles) break;
        const int last = min(first + chunk, ntiles);
        for (int t = first; t < last; ++t) {
            const EngineTile tile = tiles[t];
            const EngineSolve<C>& B = solves[tile.slot];
            const KParams<C>& k = B.k;
            if (tile.slot != cur_slot) {
                // per-plane pull bases (interior offset folded in) and store bases
                __syncthreads();
                const int cur = B.phase ^ parity;
                if (threadIdx.x < V) {
                    const int a = threadIdx.x;
                    sp[a] = static_cast<const S*>(B.f[cur]) + (long long)a * k.plane - k.off[a];
                    dp[a] = static_cast<S*>(B.f[cur ^ 1]) + (long long)a * k.plane;
                }
                __syncthreads();
                cur_slot = tile.slot;
            }
            const S* src = sp[0] + k.off[0];   // lattice base of the current state
            const int c0 = tile.cell0;
            const int cell = c0 + threadIdx.x;
            const int y0 = c0 / k.Nx;
            const int x0 = c0 - y0 * k.Nx;
            const bool fast = x0 >= k.maxex && x0 + kBlock - 1 + k.maxex < k.Nx &&
                              y0 >= k.maxey && y0 < k.Ny - k.maxey;
            const int y1 = (min(c0 + kBlock, k.ncell) - 1) / k.Nx;
            const bool rows = !fast && y0 >= k.maxey && y1 < k.Ny - k.maxey;
            if (!fast && cell >= k.ncell) continue;
            C f[V];
            if (fast) {
#pragma unroll
                for (int a = 0; a < V; ++a) f[a] = ld_pop<S, C>(k, sp[a][cell], a);
            } else if (rows || (cell / k.Nx >= k.maxey && cell / k.Nx < k.Ny - k.maxey)) {
                // nodes away from the walls (the whole tile, or this node of a wall tile)
                pull_rows_any<SET, S, C>(k, sp, cell, f);
            } else {
                const int y = cell / k.Nx;
                const int x = cell - y * k.Nx;
                const bool nb = y < k.maxey, nt = y >= k.Ny - k.maxey;
                const double pb = nb ? wall_dpsi<S, C>(k, src, x, true) : 0.0;
                const double pt = nt ? wall_dpsi<S, C>(k, src, x, false) : 0.0;
#pragma unroll
                for (int a = 0; a < V; ++a) {
                    const int ys = y - k.ey[a];
                    if (ys < 0)
                        f[a] = C(pb * k.w[a]);
                    else if (ys >= k.Ny)
                        f[a] = C(pt * k.w[a]);
                    else
                        f[a] = pull<S, C>(k, src, a, x, y);
                }
            }
            C drho = R ? f[0] : C(0), Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
            moments_ct<SET, C>(f, drho, Jx, Jy, Kxx, Kxy, Kyy, std::make_integer_sequence<int, P>{});
            const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, Kxy, Kyy);
            if (R) f[0] = fma(k.one_m_omega, f[0], k.omw_rest * q.a0);
            if (k.force)
                relax_ct<SET, N, true, C>(k, q, f, std::make_integer_sequence<int, P>{});
            else
                relax_ct<SET, N, false, C>(k, q, f, std::make_integer_sequence<int, P>{});
            unsigned rs = sr_seed<S, C>(seed + unsigned(tile.slot) * 0x632be5abu, cell);
#pragma unroll
            for (int a = 0; a < V; ++a) dp[a][cell] = st_pop<S, C>(k, f[a], a, rs);
            if (emit == 1) {
                B.rho[cell] = 1.0 + (double)q.drho;
                B.ux[cell] = (double)q.ux;
                B.uy[cell] = (double)q.uy;
            } else if (emit == 2) {
                B.prev[cell] = (double)q.ux;
            }
            flag_density<C>(q, B.status);
        }
    }
}

}  // namespace lbm

namespace lbm {

// Per-solve fp64 observables of every active slot, one block per slot:
// out[4 slot + {0, 1, 2, 3}] = {max |u_x - prev|, mdot, u_s, <u_x>}.
template <typename C>
__global__ void __launch_bounds__(256)
k_engine_reduce(const EngineSolve<C>* __restrict__ solves, const int* __restrict__ active,
                double* __restrict__ out) {
    const int slot = blockIdx.x;
    if (!active[slot]) return;
    const EngineSolve<C>& B = solves[slot];
    const KParams<C>& k = B.k;
    __shared__ double sh[8];
    __shared__ double rows[10];
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < k.ncell; i += 256) {
        const double u = B.ux[i];
        s += u;
        const double d = fabs(u - B.prev[i]);
        m = (d != d || m != m) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(m, d);
    }
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        double t = 0.0;
        if (threadIdx.x == 0)
            for (int j = 0; j < 8; ++j) t += sh[j];
        return t;
    };
    auto bmax = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = (w != w || v != v) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(v, w);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        double t = 0.0;
        if (threadIdx.x == 0)
            for (int j = 0; j < 8; ++j)
                t = (sh[j] != sh[j] || t != t) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(t, sh[j]);
        return t;
    };
    const double tot = bsum(s);
    const double mx = bmax(m);
    const int Nx = k.Nx, Ny = k.Ny, m2 = Ny / 2;
    int rl[10] = {0, 1, 2, Ny - 1, Ny - 2, Ny - 3, m2 - 2, m2 - 1, m2, m2 + 1};
    if (Ny & 1) rl[6] = rl[7] = rl[8] = rl[9] = (Ny - 1) / 2;
    for (int r = 0; r < 10; ++r) {
        double v = 0.0;
        if (Ny >= 4)
            for (int x = threadIdx.x; x < Nx; x += 256) v += B.ux[(long long)rl[r] * Nx + x];
        const double t = bsum(v);
        if (threadIdx.x == 0) rows[r] = t / Nx;
    }
    if (threadIdx.x == 0) {
        const double mean = tot / ((double)Nx * Ny);
        const double g = B.g, tau = B.tau;
        double us = __longlong_as_double(0x7ff8000000000000ll);
        if (Ny >= 4) {
            const double bot = (15.0 * rows[0] - 10.0 * rows[1] + 3.0 * rows[2]) / 8.0;
            const double top = (15.0 * rows[3] - 10.0 * rows[4] + 3.0 * rows[5]) / 8.0;
            const double uc = (Ny & 1) ? rows[8] : (9.0 * (rows[7] + rows[8]) - (rows[6] + rows[9])) / 16.0;
            us = 0.5 * (bot + top) / uc;
        }
        out[4 * slot + 0] = mx;
        out[4 * slot + 1] = g != 0.0 ? 2.0 * tau * mean / (g * B.kn) : __longlong_as_double(0x7ff8000000000000ll);
        out[4 * slot + 2] = us;
        out[4 * slot + 3] = mean;
    }
}

}  // namespace lbm
