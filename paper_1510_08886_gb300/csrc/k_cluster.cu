// Resident chunk of a tiny fp64 or fp32 channel on one thread-block cluster.
//
// A channel of a few hundred nodes cannot fill the GPU, so its per-step cost is
// launch latency plus one node's dependency chain.  This kernel runs K steps
// (Sect. V's time marching, Eq. nm.8 with the walls of Eq. nm.14/15) in one
// launch: the CTAs of one cluster split the rows of the channel, both lattices
// live in their shared memory, a population streamed across a CTA boundary is
// read from the owner's shared memory (distributed shared memory), and the
// cluster's hardware barrier separates the steps.  Each node is updated by the
// same warp_node body as k_step_warp (LP lanes per node, the same fp64
// operations in the same order) and the wall balance by the same wall_dpsi_by
// sum, so K steps here give the bits of K launches of k_step_warp.
//
// No thread leaves before the last barrier: every thread executes the same K + 1
// cluster barriers, so the barrier cannot wait on a CTA that has exited, and no
// CTA exits while another may still read its shared memory.
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Release this CTA's shared-memory writes to the cluster and wait for all CTAs.
__device__ __forceinline__ void cluster_sync() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Generic address of the object at generic shared address p in CTA r of the cluster.
template <typename T>
__device__ __forceinline__ const T* map_rank(const T* p, unsigned r) {
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(r));
    return reinterpret_cast<const T*>(out);
}

// One term of a wall flux balance (Eq. nm.15): plane b at one row, as a
// generic address of column 0 of that row in lattice 0 of the CTA that owns
// the row; sx = e_x mod Nx of plane b (the source column is x - e_x).
template <typename S>
struct WallTerm {
    const S* p0;
    int sx, b;
};

// Where a lane's population comes from in every step: pulled from a fixed
// address (kind 0; lattice 1 is lbuf elements further) or filled by the bottom
// (1) or top (2) wall, cw = its weight in the compute type.
template <typename S, typename C>
struct Source {
    const S* p0;
    int kind;
    C cw;
};

// K steps of one channel on a cluster whose CTA r holds rows [r rows,
// (r + 1) rows) of both lattices in its shared memory, [2][V][rows][Nx], and
// after them the term tables of the two walls (nb, nt terms).  One warp per
// group of 32 / LP nodes (the launch has as many warps as the largest CTA has
// groups), so each lane keeps its node, sources and pair constants in
// registers for the whole chunk.  fin: the state (global [V][Ny][Nx]); fout:
// where the state after K steps is written.  Step K - 1 (the last) writes rho,
// u_x, u_y to b; with emit_prev, step K - 2 writes u_x to b.prev_ux (the
// convergence test compares the two).
//
// The wall sums are split over the first four lanes of a wall node: lane j adds
// the terms j, j + 4, ... in order, exactly accumulator j of Acc4, and two
// shuffles form (a0 + a1) + (a2 + a3) -- the bits of wall_dpsi.
template <int LP, int N, typename S, typename C>
__global__ void __launch_bounds__(kClusterThreads)
k_chunk_cluster(const __grid_constant__ KParams<C> k, const S* fin, S* fout, const DevBufs b,
                int K, int rows, int emit_prev, int nb, int nt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = 32 / LP;
    constexpr unsigned FULL = 0xffffffffu;
    S* lat = reinterpret_cast<S*>(smem_raw);
    const long long lplane = (long long)rows * k.Nx;
    const long long lbuf = (long long)k.V * lplane;
    WallTerm<S>* tab = reinterpret_cast<WallTerm<S>*>(smem_raw + ((2 * lbuf * sizeof(S) + 15) & ~15ull));
    const unsigned rank = cluster_rank();
    const int ylo = int(rank) * rows;
    const int nloc = max(0, min(rows, k.Ny - ylo)) * k.Nx;     // nodes of this CTA
    const long long g0 = (long long)ylo * k.Nx;                // first global cell
    for (int i = threadIdx.x; i < k.V * nloc; i += blockDim.x) {
        const int a = i / nloc, c = i - a * nloc;
        lat[a * lplane + c] = fin[(long long)a * k.plane + g0 + c];
    }
    // generic address of element off of lattice 0 in the CTA owning row `row`
    auto owner = [&](int row, long long off) -> const S* {
        const unsigned r = unsigned(row / rows);
        const S* q = lat + (long long)(row - int(r) * rows) * k.Nx + off;
        return r == rank ? q : map_rank(q, r);
    };
    if (threadIdx.x == 0) {             // wall terms in the order of wall_dpsi_by
        int ib = 0, it = 0;
        for (int pl = k.R; pl < k.V; ++pl) {
            const int ey = k.ey[pl];
            for (int j = 0; j < (ey < 0 ? -ey : 0) && ib < nb; ++j, ++ib)
                tab[ib] = WallTerm<S>{owner(j, pl * lplane), k.sx[pl], pl};
            for (int j = 0; j < (ey > 0 ? ey : 0) && it < nt; ++j, ++it)
                tab[nb + it] = WallTerm<S>{owner(k.Ny - 1 - j, pl * lplane), k.sx[pl], pl};
        }
    }
    cluster_sync();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = lane % LP, lead = lane - p;
    const int cl = warp * G + lane / LP;
    const bool node = cl < nloc;
    int y = 0, x = 0;
    if (node) {
        const int yl = cl / k.Nx;
        x = cl - yl * k.Nx;
        y = ylo + yl;
    }
    const bool act = node && p < k.P;
    const bool has0 = node && p == 0 && k.R;
    const PairConst<C> pc = pair_const(k, act ? p : 0);
    auto source = [&](int a) -> Source<S, C> {
        Source<S, C> src{nullptr, 0, k.cw[a]};
        const int ys = y - k.ey[a];
        if (ys < 0) {
            src.kind = 1;
        } else if (ys >= k.Ny) {
            src.kind = 2;
        } else {
            int xs = x - k.sx[a];
            xs += (xs < 0) ? k.Nx : 0;
            src.p0 = owner(ys, a * lplane + xs);
        }
        return src;
    };
    const Source<S, C> sp = source(act ? k.R + p : 0), sm = source(act ? k.R + k.P + p : 0);
    const Source<S, C> s0 = source(0);
    const bool wb = node && y < k.maxey, wt = node && y >= k.Ny - k.maxey;
    const bool any_b = __any_sync(FULL, wb), any_t = __any_sync(FULL, wt);
    // dPsi of this lane's node and wall (term tables tab[0, n)), lattice offset to
    auto wall = [&](const WallTerm<S>* tw, int n, bool mine, long long to) -> C {
        double acc = 0.0;
        if (mine && p < 4)
            for (int i = p; i < n; i += 4) {
                int xs = x - tw[i].sx;
                xs += (xs < 0) ? k.Nx : 0;
                acc += (double)ld_pop<S, C>(k, tw[i].p0[to + xs], tw[i].b);
            }
        const double s2 = acc + __shfl_sync(FULL, acc, (lane + 1) & 31);      // a0 + a1, a2 + a3
        const double tot = s2 + __shfl_sync(FULL, s2, (lane + 2) & 31);       // on lane 0 of the node
        return C(__shfl_sync(FULL, tot * k.inv_den, lead));
    };
    auto value = [&](const Source<S, C>& src, C pb, C pt, long long to, int a) -> C {
        if (src.kind == 1) return mul_rn(pb, src.cw);
        if (src.kind == 2) return mul_rn(pt, src.cw);
        return ld_pop<S, C>(k, src.p0[to], a);
    };
    int t = 0;
    for (int s = 0; s < K; ++s) {
        const long long to = t ? lbuf : 0;
        S* dst = lat + (t ? 0 : lbuf);
        const C pb = any_b ? wall(tab, nb, wb, to) : C(0);
        const C pt = any_t ? wall(tab + nb, nt, wt, to) : C(0);
        const C fp = act ? value(sp, pb, pt, to, k.R + p) : C(0);
        const C fm = act ? value(sm, pb, pt, to, k.R + k.P + p) : C(0);
        const C f0 = has0 ? value(s0, pb, pt, to, 0) : C(0);
        auto put = [&](int a, C v) { dst[a * lplane + cl] = S(v); };
        const CellCoef<C> q = warp_node<LP, N, C>(k, p, node, pc, fp, fm, f0, put);
        if (node && p == 0) {
            if (s == K - 1) store_moments<C>(q, int(g0 + cl), b);
            else if (emit_prev && s == K - 2) b.prev_ux[g0 + cl] = (double)q.ux;
            flag_density<C>(q, b.status);
        }
        cluster_sync();
        t = 1 - t;
    }
    for (int i = threadIdx.x; i < k.V * nloc; i += blockDim.x) {
        const int a = i / nloc, c = i - a * nloc;
        fout[(long long)a * k.plane + g0 + c] = lat[t * lbuf + a * lplane + c];
    }
}

template <int LP, int N, typename C>
void* cluster_kernel() {
    return reinterpret_cast<void*>(&k_chunk_cluster<LP, N, C, C>);
}

template <typename C>
void* pick_kernel(int N, int LP) {
    switch (LP * 10 + N) {
        case 82: return cluster_kernel<8, 2, C>();
        case 83: return cluster_kernel<8, 3, C>();
        case 84: return cluster_kernel<8, 4, C>();
        case 162: return cluster_kernel<16, 2, C>();
        case 163: return cluster_kernel<16, 3, C>();
        case 164: return cluster_kernel<16, 4, C>();
        case 322: return cluster_kernel<32, 2, C>();
        case 323: return cluster_kernel<32, 3, C>();
        case 324: return cluster_kernel<32, 4, C>();
        default: return nullptr;
    }
}

cudaLaunchConfig_t cluster_config(const ClusterPlan& pl, cudaStream_t st, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.ctas);
    cfg.blockDim = dim3(pl.threads);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = pl.ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

// Choose the cluster for a channel (fp64 or fp32 storage and arithmetic, C)
// whose step runs on LP lanes per node:
// the rows split evenly over at most 16 CTAs (8 where 16 cannot be placed), at
// most kClusterThreads / 32 warps per CTA, shared memory padded so that each CTA
// has an SM (and its fp64 lanes) of its own.  pl.ctas = 0: not resident.
template <typename C>
int plan_cluster_t(const KParams<C>& k, int N, int LP, ClusterPlan& pl) {
    pl = ClusterPlan{};
    void* fn = pick_kernel<C>(N, LP);
    if (!fn) return 0;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int G = 32 / LP;
    int nb = 0, nt = 0;                      // wall terms (Eq. nm.15 sums)
    for (int a = k.R; a < k.V; ++a) {
        if (k.ey[a] < 0) nb += -k.ey[a];
        if (k.ey[a] > 0) nt += k.ey[a];
    }
    for (int cmax : {16, 8}) {
        const int rows = (k.Ny + cmax - 1) / cmax;
        const int ctas = (k.Ny + rows - 1) / rows;
        const int groups = (rows * k.Nx + G - 1) / G;      // warps of work per CTA
        if (groups > kClusterThreads / 32) continue;
        const size_t need = ((size_t(2) * k.V * rows * k.Nx * sizeof(C) + 15) & ~size_t(15)) +
                            size_t(nb + nt) * sizeof(WallTerm<C>);
        const size_t smem = std::max(need, size_t(kClusterSmemPad));
        if (smem > size_t(optin)) continue;
        ClusterPlan c;
        c.ctas = ctas;
        c.rows = rows;
        c.threads = 32 * groups;
        c.smem = smem;
        c.N = N;
        c.LP = LP;
        c.nb = nb;
        c.nt = nt;
        // the limit is per kernel and shared by every solver that uses it: set it
        // to the device's maximum, so that a later, smaller plan cannot lower it
        // below what an earlier solver's launches need
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
                cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaLaunchAttribute at[1];
        const cudaLaunchConfig_t cfg = cluster_config(c, nullptr, at);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters < 1) continue;
        pl = c;
        return 1;
    }
    return 0;
}

template <typename C>
cudaError_t launch_chunk_cluster_t(const KParams<C>& k, const ClusterPlan& pl, const void* fin,
                                   void* fout, const DevBufs& b, int K, bool emit_prev,
                                   cudaStream_t st) {
    void* fn = pick_kernel<C>(pl.N, pl.LP);
    if (!fn || pl.ctas < 1 || K < 1) return cudaErrorInvalidValue;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = cluster_config(pl, st, at);
    const C* src = static_cast<const C*>(fin);
    C* dst = static_cast<C*>(fout);
    int rows = pl.rows, ep = emit_prev ? 1 : 0, nb = pl.nb, nt = pl.nt;
    void* args[] = {const_cast<KParams<C>*>(&k), &src, &dst, const_cast<DevBufs*>(&b),
                    &K, &rows, &ep, &nb, &nt};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int plan_cluster(const KParams<double>& k, int N, int LP, ClusterPlan& pl) {
    return plan_cluster_t(k, N, LP, pl);
}
int plan_cluster(const KParams<float>& k, int N, int LP, ClusterPlan& pl) {
    return plan_cluster_t(k, N, LP, pl);
}
cudaError_t launch_chunk_cluster(const KParams<double>& k, const ClusterPlan& pl, const void* fin,
                                 void* fout, const DevBufs& b, int K, bool emit_prev,
                                 cudaStream_t st) {
    return launch_chunk_cluster_t(k, pl, fin, fout, b, K, emit_prev, st);
}
cudaError_t launch_chunk_cluster(const KParams<float>& k, const ClusterPlan& pl, const void* fin,
                                 void* fout, const DevBufs& b, int K, bool emit_prev,
                                 cudaStream_t st) {
    return launch_chunk_cluster_t(k, pl, fin, fout, b, K, emit_prev, st);
}

}  // namespace lbm
