// Device code of the multi-solve engine: one time step of many independent
// channels in one persistent launch per compiled velocity set.
//
// Work is a list of tiles (solve slot, first node, shape) of one channel:
// m kBlock consecutive nodes, or a rectangle of tw columns x m kBlock / tw
// rows.  Blocks of a fixed, SM-filling grid take `chunk` tiles at a time from
// an atomic counter, so small and large channels, wall tiles and interior
// tiles balance across the GPU.  Each tile runs the same
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

// A tile: m = 2^lm sub-tiles of kBlock nodes of one channel (m = 1, 2 or 4,
// the same for every tile of a launch).  Linear tiles (tws = 0) are m kBlock
// consecutive nodes from cell0 in row-major order, sub-tile j the j-th run of
// kBlock; 2-D tiles (tws = 5, 6 or 7: width tw = 2^tws columns, Nx a multiple
// of tw) are tw columns x m kBlock / tw rows from node cell0 = y0 Nx + x0,
// sub-tile j the j-th band of kBlock / tw rows.  Thread i of the block
// updates node i of each sub-tile (column x0 + i mod tw of a 2-D tile).  The
// shape only changes which block updates a node, never the node's arithmetic.
struct EngineTile {
    int slot;
    int cell0;
    int tws;
};

// Registers per thread allowed beyond the populations' share (min_blocks_for),
// chosen per set from ptxas's spill report and measured throughput: with the
// solve's constants read from shared memory the 53-velocity set fits 96
// registers (20 warps per SM); the 48-velocity set spills there and keeps 24
// extra, the 40-velocity set 12; sets of at most 16 pairs take 6 (the
// 33-velocity set at 72 registers, 28 warps per SM, a 16-byte spill: 3 %
// faster than 80 registers without one).
template <class SET>
constexpr int engine_extra_regs() {
    return SET::R + 2 * SET::P == 53 ? 0 : (SET::P > 20 ? 24 : (SET::P > 16 ? 12 : 6));
}

// Moments, equilibrium, force and relaxation of one node (register values
// f in place): the arithmetic of k_step_ct, shared by both engine kernels.
template <class SET, int N, typename S, typename C>
__device__ __forceinline__ CellCoef<C> res_collide(const KParams<C>& k, C* f) {
    C drho, Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
    moments_ct<SET, S, C>(k, f, drho, Jx, Jy, Kxx, Kxy, Kyy, std::make_integer_sequence<int, SET::P>{});
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, Kxy, Kyy);
    relax_ct<SET, N, S, C>(k, q, f);
    return q;
}

// Copy the parts of a solve's constants that kernels of a compiled set read:
// the scalars and the first V (per plane) or P (per pair) entries of every
// array; the arrays are sized for LBM_MAX_V, so this moves about a third of
// the record.
template <class SET, typename C>
__device__ __forceinline__ void copy_params(const KParams<C>& src, KParams<C>& dst) {
    using K = KParams<C>;
    constexpr int V = SET::R + 2 * SET::P, P = SET::P;
    constexpr int cv = int(sizeof(C) / 4) * V, cp = int(sizeof(C) / 4) * P;
    // (first 4-byte word, words)
    constexpr int seg[][2] = {
        {0, int(offsetof(K, ex) / 4)},
        {int(offsetof(K, ex) / 4), V}, {int(offsetof(K, ey) / 4), V}, {int(offsetof(K, sx) / 4), V},
        {int(offsetof(K, off) / 4), V}, {int(offsetof(K, dx) / 4), V},
        {int(offsetof(K, srcf) / 4), 2 * V}, {int(offsetof(K, dstp) / 4), 2 * V},
        {int(offsetof(K, w) / 4), 2 * V},
        {int(offsetof(K, cw) / 4), cv}, {int(offsetof(K, sw) / 4), cv}, {int(offsetof(K, isw) / 4), cv},
        {int(offsetof(K, hw) / 4), cp}, {int(offsetof(K, hwx) / 4), cp}, {int(offsetof(K, hwy) / 4), cp},
        {int(offsetof(K, hwxx) / 4), cp}, {int(offsetof(K, hwxy) / 4), cp}, {int(offsetof(K, hwyy) / 4), cp},
        {int(offsetof(K, hw_rest) / 4), int((offsetof(K, pex) - offsetof(K, hw_rest)) / 4)},
        {int(offsetof(K, pex) / 4), cp}, {int(offsetof(K, pey) / 4), cp}, {int(offsetof(K, pexx) / 4), cp},
        {int(offsetof(K, pexy2) / 4), cp}, {int(offsetof(K, peyy) / 4), cp}, {int(offsetof(K, pge) / 4), cp},
        {int(offsetof(K, pomw) / 4), cp},
        {int(offsetof(K, omw_rest) / 4), int((sizeof(K) - offsetof(K, omw_rest)) / 4)}};
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
#pragma unroll
    for (int g = 0; g < int(sizeof(seg) / sizeof(seg[0])); ++g)
        for (int i = int(threadIdx.x); i < seg[g][1]; i += kBlock) d[seg[g][0] + i] = s[seg[g][0] + i];
}

// emit: 0 = nothing, 1 = rho, u_x, u_y into the moment fields, 2 = u_x into prev
template <class SET, int N, typename S, typename C>
__global__ void __launch_bounds__(kBlock, min_blocks_for(SET::R + 2 * SET::P + engine_extra_regs<SET>(),
                                                         sizeof(C)))
k_engine_step(const EngineSolve<C>* __restrict__ solves, const EngineTile* __restrict__ tiles,
              const int* __restrict__ ntiles_p, const int* __restrict__ tile_off_p,
              int* __restrict__ counter,
              const unsigned int* __restrict__ seed_p, int parity, int emit, int chunk, int lm) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P;
    __shared__ const S* sp[V];
    __shared__ S* dp[V];
    __shared__ int s_first[2];
    __shared__ KParams<C> s_k;
    const int ntiles = *ntiles_p;
    tiles += *tile_off_p;
    const unsigned seed = *seed_p + unsigned(parity);
    int cur_slot = -1;
    // One barrier per grab: every thread reads grab i's first tile from
    // s_first[i & 1] before it reaches the barrier of grab i + 1, after which
    // thread 0 may overwrite that entry (at grab i + 2).
    for (int it = 0;; ++it) {
        if (threadIdx.x == 0) s_first[it & 1] = atomicAdd(counter, chunk);
        __syncthreads();
        const int first = s_first[it & 1];
        if (first >= ntiles) break;
        const int last = min(first + chunk, ntiles);
        // sub-tiles u of the tiles [first, last)
        for (int u = first << lm; u < (last << lm); ++u) {
            const EngineTile tile = tiles[u >> lm];
            const int j = u & ((1 << lm) - 1);
            const EngineSolve<C>& B = solves[tile.slot];
            const KParams<C>& k = s_k;
            if (tile.slot != cur_slot) {
                // The previous slot's constants and plane bases are free once
                // every thread is past its last sub-tile: at the grab's
                // barrier for the grab's first sub-tile, else at this one.
                if (u != (first << lm)) __syncthreads();
                copy_params<SET, C>(B.k, s_k);
                // per-plane pull bases (interior offset folded in) and store bases
                const int cur = B.phase ^ parity;
                if (threadIdx.x < V) {
                    const int a = threadIdx.x;
                    const long long plane = B.k.plane;
                    sp[a] = static_cast<const S*>(B.f[cur]) + (long long)a * plane - B.k.off[a];
                    dp[a] = static_cast<S*>(B.f[cur ^ 1]) + (long long)a * plane;
                }
                __syncthreads();
                cur_slot = tile.slot;
            }
            const S* src = sp[0] + k.off[0];   // lattice base of the current state
            // node of this thread in sub-tile j; fast = every node of the
            // sub-tile pulls at fixed offsets; rows = no node is near a wall
            int cell, ya, yb;
            bool fast;
            if (tile.tws == 0) {
                const int cs = tile.cell0 + j * kBlock;
                cell = cs + int(threadIdx.x);
                ya = cs / k.Nx;
                const int xa = cs - ya * k.Nx;
                yb = (min(cs + kBlock, k.ncell) - 1) / k.Nx;
                fast = xa >= k.maxex && xa + kBlock - 1 + k.maxex < k.Nx && ya >= k.maxey &&
                       ya < k.Ny - k.maxey;
            } else {
                const int tws = tile.tws;
                const int y0 = tile.cell0 / k.Nx;
                const int x0 = tile.cell0 - y0 * k.Nx;
                ya = y0 + j * (kBlock >> tws);              // kBlock / tw rows per sub-tile
                yb = min(ya + (kBlock >> tws), k.Ny) - 1;
                cell = (ya + (int(threadIdx.x) >> tws)) * k.Nx + x0 + (int(threadIdx.x) & ((1 << tws) - 1));
                fast = x0 >= k.maxex && x0 + (1 << tws) - 1 + k.maxex < k.Nx && ya >= k.maxey &&
                       ya + (kBlock >> tws) - 1 < k.Ny - k.maxey;
            }
            // a node beyond the channel (cell >= ncell: past the last node, or
            // a row at or above Ny of a 2-D tile) has nothing to do
            if (!fast && cell >= k.ncell) continue;
            const bool rows = !fast && ya >= k.maxey && yb < k.Ny - k.maxey;
            C f[V];
            if (fast) {
#pragma unroll
                for (int a = 0; a < V; ++a) f[a] = ld_val<S, C>(ld_stream(sp[a] + cell));
            } else if (rows || (cell / k.Nx >= k.maxey && cell / k.Nx < k.Ny - k.maxey)) {
                // nodes away from the walls (the whole sub-tile, or this node of a wall tile)
                pull_rows_any<SET, S, C>(k, sp, cell, f);
            } else {
                const int y = cell / k.Nx;
                const int x = cell - y * k.Nx;
                pull_wall_ct<SET, S, C>(k, src, x, y, f, std::make_integer_sequence<int, V>{});
            }
            const CellCoef<C> q = res_collide<SET, N, S, C>(k, f);
            S out[V];
            pack_ct<SET, S, C>(f, sr_seed<S, C>(seed + unsigned(tile.slot) * 0x632be5abu, cell), out);
#pragma unroll
            for (int a = 0; a < V; ++a) dp[a][cell] = out[a];
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

// ---- resident chunks ----------------------------------------------------------
// Channels small enough for shared memory run a whole chunk of K steps there:
// one block loads a bundle of such channels once, advances them K steps with
// one barrier per step, and writes the state back once.  Streaming is in
// place with the two-step (A/B) pattern on the +-e pairs: in a B step node n
// reads population a from slot (n - e_a, abar) and writes its post-collision
// value to (n + e_a, a); in an A step it reads (n, a) and writes (n, abar).
// Each node's read set equals its write set, so no node overwrites a value
// another node still has to read.  Populations that leave through a wall in a
// B step land in maxey ghost rows beyond the wall, where the next A step's
// flux balance (Eq. nm.15) finds them; in a B step the leaving populations
// of the previous A step sit untouched in their source nodes.  Loads, fills,
// moment sums, relaxation and roundings are those of k_engine_step, in the
// same order, so the results are bitwise those of the tiled kernel.

constexpr int kResMaxCh = 64;      // channels per bundle
constexpr int kResNodes = 4096;    // padded nodes per bundle (channels start at multiples of 32)

struct ResChannel {
    int slot;
    int start;      // first node in the bundle's node numbering (a multiple of 32)
    int off;        // element offset of the channel's planes in shared memory
    int ncell;
};

struct ResBundle {
    int first;      // channels [first, first + count) of the channel list
    int count;
    int nodes;      // padded node count
    int pad;
};

template <class SET>
__host__ __device__ constexpr int plane_ey(int a) {
    return a < SET::R ? 0 : (a < SET::R + SET::P ? SET::ey[a - SET::R] : -SET::ey[a - SET::R - SET::P]);
}

template <class SET>
__host__ __device__ constexpr int plane_opp(int a) {
    return a < SET::R ? a : (a < SET::R + SET::P ? a + SET::P : a - SET::P);
}

template <class SET>
__host__ __device__ constexpr int set_maxey() {
    int m = 0;
    for (int p = 0; p < SET::P; ++p) m = SET::ey[p] > m ? SET::ey[p] : (-SET::ey[p] > m ? -SET::ey[p] : m);
    return m;
}

// Threads of a resident block: the V populations of a node stay in
// registers, so fp64 (two registers a value) halves the block.
template <class SET, typename C = float>
__host__ __device__ constexpr int res_threads() {
    return (SET::R + 2 * SET::P <= 16 ? 1024 : 512) / (sizeof(C) == 8 ? 2 : 1);
}

// (x + d) mod Nx for x in [0, Nx); mode 0: Nx = 1, 1: Nx >= |d|, 2: any Nx
template <int D, int MODE>
__device__ __forceinline__ int xwrap(int x, int Nx) {
    if constexpr (D == 0 || MODE == 0) {
        return MODE == 0 ? 0 : x;
    } else if constexpr (MODE == 1) {
        const int t = x + D;
        if constexpr (D > 0) return t >= Nx ? t - Nx : t;
        else return t < 0 ? t + Nx : t;
    } else {
        const int t = (x + D) % Nx;
        return t < 0 ? t + Nx : t;
    }
}

// Flux balance of Eq. nm.15 for landing column x from shared memory: the
// same terms, in the same order, as wall_dpsi.  In a B step the leaving
// population b of node m = (x - e_x, j) sits at (m, bbar); in an A step it
// sits in the ghost row at (m + e_b, b).
template <class SET, typename S, typename C, bool BOTTOM, bool STEP_A>
__device__ __forceinline__ double res_wall_dpsi(const KParams<C>& k, const S* sb, int PS, int x) {
    constexpr int V = SET::R + 2 * SET::P, G = set_maxey<SET>();
    const int Nx = k.Nx;
    auto term = [&](auto bc, int j) {
        constexpr int b = decltype(bc)::value;
        const int row = BOTTOM ? j : (k.Ny - 1 - j);
        S v;
        if (STEP_A) {
            v = sb[b * PS + (row + plane_ey<SET>(b) + G) * Nx + x];
        } else {
            int xs = x - k.sx[b];
            xs += (xs < 0) ? Nx : 0;
            v = sb[plane_opp<SET>(b) * PS + (row + G) * Nx + xs];
        }
        return (double)ld_pop<S, C>(k, v, b);
    };
    return wall_sum_ct<SET, BOTTOM>(term, std::make_integer_sequence<int, V>{}) * k.inv_den;
}

// Population A of a wall node from shared memory (fill or in-domain value).
template <class SET, typename S, typename C, bool STEP_A, int A>
__device__ __forceinline__ C res_wall_value(const KParams<C>& k, const S* sb, int PS, int x, int y,
                                            C pb, C pt) {
    constexpr int G = set_maxey<SET>();
    constexpr int EY = plane_ey<SET>(A);
    const int Nx = k.Nx;
    const int ys = y - EY;
    if (ys < 0) return fill_val<S, C>(k, pb, A);
    if (ys >= k.Ny) return fill_val<S, C>(k, pt, A);
    if (STEP_A) return ld_val<S, C>(sb[A * PS + (y + G) * Nx + x]);
    int xs = x - k.sx[A];
    xs += (xs < 0) ? Nx : 0;
    return ld_val<S, C>(sb[plane_opp<SET>(A) * PS + (ys + G) * Nx + xs]);
}

template <class SET, typename S, typename C, bool STEP_A, int... I>
__device__ __forceinline__ void res_pull_wall(const KParams<C>& k, const S* sb, int PS, int x, int y,
                                              C* f, std::integer_sequence<int, I...>) {
    constexpr int G = set_maxey<SET>();
    const C pb = y < G ? C(res_wall_dpsi<SET, S, C, true, STEP_A>(k, sb, PS, x)) : C(0);
    const C pt = y >= k.Ny - G ? C(res_wall_dpsi<SET, S, C, false, STEP_A>(k, sb, PS, x)) : C(0);
    ((f[I] = res_wall_value<SET, S, C, STEP_A, I>(k, sb, PS, x, y, pb, pt)), ...);
}

template <class SET, typename S, typename C, int MODE, bool STEP_A, int... I>
__device__ __forceinline__ void res_pull(const KParams<C>& k, const S* sb, int PS, int x, int y,
                                         C* f, std::integer_sequence<int, I...>) {
    constexpr int G = set_maxey<SET>();
    const int Nx = k.Nx;
    if constexpr (STEP_A) {
        const int o = (y + G) * Nx + x;
        ((f[I] = ld_val<S, C>(sb[I * PS + o])), ...);
    } else {
        ((f[I] = ld_val<S, C>(sb[plane_opp<SET>(I) * PS + (y - plane_ey<SET>(I) + G) * Nx +
                                 xwrap<-plane_ex<SET>(I), MODE>(x, Nx)])), ...);
    }
}

template <class SET, typename S, typename C, int MODE, bool STEP_A, int... I>
__device__ __forceinline__ void res_push(const KParams<C>& k, S* sb, int PS, int x, int y, const C* f,
                                         unsigned rs, std::integer_sequence<int, I...>) {
    constexpr int G = set_maxey<SET>();
    const int Nx = k.Nx;
    S out[sizeof...(I)];
    pack_ct<SET, S, C>(f, rs, out);
    if constexpr (STEP_A) {
        const int o = (y + G) * Nx + x;
        ((sb[plane_opp<SET>(I) * PS + o] = out[I]), ...);
    } else {
        ((sb[I * PS + (y + plane_ey<SET>(I) + G) * Nx + xwrap<plane_ex<SET>(I), MODE>(x, Nx)] =
              out[I]), ...);
    }
}

template <typename C>
__device__ __forceinline__ void res_emit(const EngineSolve<C>& B, const CellCoef<C>& q, int cell,
                                         int emit) {
    if (emit == 1) {
        B.rho[cell] = 1.0 + (double)q.drho;
        B.ux[cell] = (double)q.ux;
        B.uy[cell] = (double)q.uy;
    } else if (emit == 2) {
        B.prev[cell] = (double)q.ux;
    }
    flag_density<C>(q, B.status);
}

// One node of one A or B step.  sb: the channel's planes (PS elements each,
// row y of the channel at row y + G of a plane).
template <class SET, int N, typename S, typename C, bool STEP_A>
__device__ __forceinline__ void res_node(const EngineSolve<C>& B, S* sb, int PS, int slot, int cell,
                                         unsigned seed, int emit) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P, G = set_maxey<SET>();
    const KParams<C>& k = B.k;
    const int Nx = k.Nx, Ny = k.Ny;
    const int y = Nx == 1 ? cell : cell / Nx;     // one-column channels need no division
    const int x = cell - y * Nx;
    C f[V];
    const int mode = Nx == 1 ? 0 : (Nx >= k.maxex ? 1 : 2);
    if (y >= G && y < Ny - G) {
        if (mode == 0)
            res_pull<SET, S, C, 0, STEP_A>(k, sb, PS, x, y, f, std::make_integer_sequence<int, V>{});
        else if (mode == 1)
            res_pull<SET, S, C, 1, STEP_A>(k, sb, PS, x, y, f, std::make_integer_sequence<int, V>{});
        else
            res_pull<SET, S, C, 2, STEP_A>(k, sb, PS, x, y, f, std::make_integer_sequence<int, V>{});
    } else {
        res_pull_wall<SET, S, C, STEP_A>(k, sb, PS, x, y, f, std::make_integer_sequence<int, V>{});
    }
    const CellCoef<C> q = res_collide<SET, N, S, C>(k, f);
    const unsigned rs = sr_seed<S, C>(seed + unsigned(slot) * 0x632be5abu, cell);
    if (mode == 0)
        res_push<SET, S, C, 0, STEP_A>(k, sb, PS, x, y, f, rs, std::make_integer_sequence<int, V>{});
    else if (mode == 1)
        res_push<SET, S, C, 1, STEP_A>(k, sb, PS, x, y, f, rs, std::make_integer_sequence<int, V>{});
    else
        res_push<SET, S, C, 2, STEP_A>(k, sb, PS, x, y, f, rs, std::make_integer_sequence<int, V>{});
    res_emit<C>(B, q, cell, emit);
}

// Persistent blocks (one per SM) take bundles from an atomic counter; each
// bundle runs K (even) steps: B, A, B, A, ...  Step i uses the seed and the
// emit flags of step i of the tiled chunk.
template <class SET, int N, typename S, typename C>
__global__ void __launch_bounds__(res_threads<SET, C>(), 1)
k_engine_resident(const EngineSolve<C>* __restrict__ solves, const ResBundle* __restrict__ bundles,
                  const ResChannel* __restrict__ chans, const int* __restrict__ nbundles_p,
                  const int* __restrict__ bundle_off_p, int* __restrict__ counter,
                  const unsigned* __restrict__ seed_p, int K) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P, G = set_maxey<SET>();
    constexpr int BT = res_threads<SET, C>();
    constexpr int NPT = kResNodes / BT;
    extern __shared__ __align__(16) unsigned char res_smem[];
    S* const sm = reinterpret_cast<S*>(res_smem);
    __shared__ ResChannel sch[kResMaxCh];
    __shared__ int wch[kResNodes / 32];     // channel of each run of 32 nodes, -1: padding
    __shared__ int s_b;
    __shared__ int s_run[2];                 // per-step work counters
    const int nb = *nbundles_p;
    bundles += *bundle_off_p;
    const unsigned seed0 = *seed_p;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_b = atomicAdd(counter, 1);
        __syncthreads();
        const int bi = s_b;
        if (bi >= nb) break;
        const ResBundle bd = bundles[bi];
        for (int c = threadIdx.x; c < bd.count; c += BT) sch[c] = chans[bd.first + c];
        for (int w = threadIdx.x; w < kResNodes / 32; w += BT) wch[w] = -1;
        if (threadIdx.x == 0) s_run[0] = 0;
        __syncthreads();
        for (int c = threadIdx.x; c < bd.count; c += BT)
            for (int w = sch[c].start >> 5; w < (sch[c].start + sch[c].ncell + 31) >> 5; ++w) wch[w] = c;
        __syncthreads();
        // load: the state (post-collision values at their own nodes) goes to
        // the opposite planes, as an A step leaves it
#pragma unroll 1
        for (int j = 0; j < NPT; ++j) {
            const int g = threadIdx.x + j * BT;
            if (g >= bd.nodes) break;
            const int c = wch[g >> 5];
            if (c < 0) continue;
            const ResChannel ch = sch[c];
            const int cell = g - ch.start;
            if (cell >= ch.ncell) continue;
            const EngineSolve<C>& B = solves[ch.slot];
            const int Nx = B.k.Nx, PS = Nx * (B.k.Ny + 2 * G);
            const int y = Nx == 1 ? cell : cell / Nx, x = cell - y * Nx;
            const S* src = static_cast<const S*>(B.f[B.phase]);
            S* sb = sm + ch.off;
#pragma unroll
            for (int a = 0; a < V; ++a)
                sb[plane_opp<SET>(a) * PS + (y + G) * Nx + x] = src[(long long)a * B.k.plane + cell];
        }
        __syncthreads();
        // Each step, warps take runs of 32 nodes from a shared counter, so warps
        // that drew wall nodes or a lighter share do not hold the others at the
        // barrier.  Step i uses counter i & 1; the other one, last used in step
        // i - 1 (finished at the barrier), is reset for step i + 1.
        const int nruns = bd.nodes >> 5;
        const int lane = threadIdx.x & 31;
#pragma unroll 1
        for (int i = 0; i < K; ++i) {
            const unsigned seed = seed0 + unsigned(i & 1);
            const int emit = i == K - 1 ? 1 : (i == K - 2 ? 2 : 0);
            if (threadIdx.x == 0) s_run[(i + 1) & 1] = 0;
#pragma unroll 1
            for (;;) {
                int run = 0;
                if (lane == 0) run = atomicAdd(&s_run[i & 1], 1);
                run = __shfl_sync(0xffffffffu, run, 0);
                if (run >= nruns) break;
                const int c = wch[run];
                if (c < 0) continue;
                const ResChannel ch = sch[c];
                const int cell = run * 32 + lane - ch.start;
                if (cell < ch.ncell) {
                    const EngineSolve<C>& B = solves[ch.slot];
                    const int PS = B.k.Nx * (B.k.Ny + 2 * G);
                    if (i & 1)
                        res_node<SET, N, S, C, true>(B, sm + ch.off, PS, ch.slot, cell, seed, emit);
                    else
                        res_node<SET, N, S, C, false>(B, sm + ch.off, PS, ch.slot, cell, seed, emit);
                }
            }
            __syncthreads();
        }
        // store: after the final A step population a of node n is at (n, abar)
#pragma unroll 1
        for (int j = 0; j < NPT; ++j) {
            const int g = threadIdx.x + j * BT;
            if (g >= bd.nodes) break;
            const int c = wch[g >> 5];
            if (c < 0) continue;
            const ResChannel ch = sch[c];
            const int cell = g - ch.start;
            if (cell >= ch.ncell) continue;
            const EngineSolve<C>& B = solves[ch.slot];
            const int Nx = B.k.Nx, PS = Nx * (B.k.Ny + 2 * G);
            const int y = Nx == 1 ? cell : cell / Nx, x = cell - y * Nx;
            S* dst = static_cast<S*>(B.f[B.phase]);
            const S* sb = sm + ch.off;
#pragma unroll
            for (int a = 0; a < V; ++a)
                dst[(long long)a * B.k.plane + cell] = sb[plane_opp<SET>(a) * PS + (y + G) * Nx + x];
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
