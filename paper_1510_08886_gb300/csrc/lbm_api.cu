// Host implementation of the C ABI declared in include/lbm.h: solver set-up
// and validation, workspace layout, the time-step loop, the steady-state
// driver, the fp64 reductions (mass flow, slip velocity, convergence test)
// and checkpoint / resume.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dvm_sets.h"
#include "lbm.h"
#include "lbm_internal.h"

using lbm::DevBufs;
using lbm::KParams;

struct lbm_solver : lbm::SolveSpec {
    cudaStream_t stream = nullptr;
    bool owns = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    DevBufs b{};
    int cur = 0;
    long steps = 0;
    KParams<double> k64{};
    KParams<float> k32{};
    // run_to_steady chunks captured as CUDA graphs, one per starting lattice
    cudaGraphExec_t chunk_exec[2] = {nullptr, nullptr};
    long chunk_K[2] = {0, 0};
    // tiny fp64 / fp32 channels: chunks of steps resident on one thread-block cluster
    lbm::ClusterPlan cl{};
    bool resident = true;
};

namespace lbm {
size_t elem_bytes(int precision) {
    return precision == LBM_FP64 ? 8 : precision == LBM_FP32 ? 4 : 2;
}
}  // namespace lbm

using lbm::elem_bytes;

namespace {

constexpr unsigned kStateMagic = 0x4c424d31u;   // "LBM1"

struct StateHeader {
    unsigned magic;
    int precision, V, Nx, Ny, N;
    long steps;
    double scale;
};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }


bool valid_precision(int p) { return p >= LBM_FP64 && p <= LBM_BF16; }
bool is16(int p) { return p == LBM_FP16 || p == LBM_BF16; }

struct Layout {
    size_t f0, f1, rho, ux, uy, prev, partial, results, status, total;
};

Layout layout(int V, size_t ncell, size_t elem) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = align256(off + n); return o; };
    L.f0 = take(size_t(V) * ncell * elem);
    L.f1 = take(size_t(V) * ncell * elem);
    L.rho = take(ncell * 8);
    L.ux = take(ncell * 8);
    L.uy = take(ncell * 8);
    L.prev = take(ncell * 8);
    L.partial = take(2 * lbm::kReduceBlocks * 8);
    L.results = take(8 * 8);
    L.status = take(256);
    L.total = off;
    return L;
}

// Velocity sets with compiled kernels, in the kernel dispatch order.
struct CompiledSet {
    int R, P;
    const int* ex;
    const int* ey;
};
template <class SET>
constexpr CompiledSet compiled() { return {SET::R, SET::P, SET::ex, SET::ey}; }
const CompiledSet kSets[] = {compiled<lbm::SetD2V16>(), compiled<lbm::SetD2V32>(),
                             compiled<lbm::SetD2V33>(), compiled<lbm::SetD2V53>(),
                             compiled<lbm::SetD2V40>(), compiled<lbm::SetD2V48>()};

// If the velocity set equals a compiled one, reorder the pairs into its order
// and return its index; else -1.
int match_compiled(const lbm_dvm* d, int R, std::vector<int>& pos, std::vector<int>& neg) {
    for (int id = 0; id < int(sizeof(kSets) / sizeof(kSets[0])); ++id) {
        const CompiledSet& cs = kSets[id];
        if (cs.R != R || cs.P != int(pos.size())) continue;
        std::vector<int> np, nn;
        for (int i = 0; i < cs.P; ++i) {
            for (size_t j = 0; j < pos.size(); ++j)
                if (d->e[2 * pos[j]] == cs.ex[i] && d->e[2 * pos[j] + 1] == cs.ey[i]) {
                    np.push_back(pos[j]);
                    nn.push_back(neg[j]);
                    break;
                }
        }
        if (int(np.size()) == cs.P) {
            pos.swap(np);
            neg.swap(nn);
            return id;
        }
    }
    return -1;
}

// Validate the DVM and put it into pair order: rest plane first (if any),
// then one member of each +-e pair, then the negatives in the same order.
int canonicalize(const lbm_dvm* d, std::vector<int>& ex, std::vector<int>& ey,
                 std::vector<double>& w, std::vector<int>& perm, int& R, int& P, int& set_id) {
    if (!d || d->D != 2 || d->V < 1 || d->V > LBM_MAX_V || !d->e || !d->w) return LBM_EINVAL;
    if (!(d->c > 0) || !std::isfinite(d->c)) return LBM_EINVAL;
    const int V = d->V;
    double sw = 0;
    for (int a = 0; a < V; ++a) {
        if (!(d->w[a] > 0) || !std::isfinite(d->w[a])) return LBM_EINVAL;
        sw += d->w[a];
        for (int b = 0; b < a; ++b)
            if (d->e[2 * a] == d->e[2 * b] && d->e[2 * a + 1] == d->e[2 * b + 1]) return LBM_EINVAL;
    }
    if (std::fabs(sw - 1.0) > 1e-12) return LBM_EINVAL;
    std::vector<int> rest, pos, neg;
    for (int a = 0; a < V; ++a) {
        const int x = d->e[2 * a], y = d->e[2 * a + 1];
        if (x == 0 && y == 0) { rest.push_back(a); continue; }
        if (!(y > 0 || (y == 0 && x > 0))) continue;
        int m = -1;
        for (int b = 0; b < V; ++b)
            if (d->e[2 * b] == -x && d->e[2 * b + 1] == -y) m = b;
        if (m < 0) return LBM_EINVAL;
        if (std::fabs(d->w[m] - d->w[a]) > 1e-13 * d->w[a]) return LBM_EINVAL;
        pos.push_back(a);
        neg.push_back(m);
    }
    if (rest.size() > 1 || rest.size() + 2 * pos.size() != size_t(V)) return LBM_EINVAL;
    R = int(rest.size());
    P = int(pos.size());
    set_id = match_compiled(d, R, pos, neg);
    perm.clear();
    for (int a : rest) perm.push_back(a);
    for (int a : pos) perm.push_back(a);
    for (int a : neg) perm.push_back(a);
    ex.resize(V);
    ey.resize(V);
    w.resize(V);
    for (int i = 0; i < V; ++i) {
        ex[i] = d->e[2 * perm[i]];
        ey[i] = d->e[2 * perm[i] + 1];
        w[i] = d->w[perm[i]];
    }
    // a pair carries one weight: the two members agree to 1e-13 (checked)
    for (int p = 0; p < P; ++p) {
        const double m = 0.5 * (w[R + p] + w[R + P + p]);
        w[R + p] = w[R + P + p] = m;
    }
    return LBM_OK;
}

template <typename C>
void fill_params_impl(const lbm::SolveSpec* s, KParams<C>& k) {
    std::memset(&k, 0, sizeof(k));
    k.Nx = s->Nx;
    k.Ny = s->Ny;
    k.ncell = s->Nx * s->Ny;
    k.R = s->R;
    k.P = s->P;
    k.V = s->V;
    k.maxey = s->maxey;
    k.maxex = s->maxex;
    k.set_id = s->set_id;
    k.force = s->g != 0.0;
    // k_step_ct's wall strips: four wall rows per wall (compiled sets with
    // max|e_y| = 4), whole blocks per row, no row within reach of both walls
    k.strips = (s->set_id >= 0 && s->maxey == 4 && s->Nx % 128 == 0 && s->Ny >= 8) ? s->Nx / 32 : 0;
    k.emit = 0;
    k.plane = (long long)s->Nx * s->Ny;
    const double omega = s->dt / (s->tau + 0.5 * s->dt);   // Eq. nm.8
    for (int a = 0; a < s->V; ++a) {
        k.ex[a] = s->ex[a];
        k.ey[a] = s->ey[a];
        k.sx[a] = ((s->ex[a] % s->Nx) + s->Nx) % s->Nx;
        k.off[a] = s->ey[a] * s->Nx + s->ex[a];
        k.dx[a] = s->ex[a] - k.sx[a];
        k.w[a] = s->w[a];
        k.cw[a] = C(s->w[a]);
        k.sw[a] = C(s->w[a] * s->scale);
        k.isw[a] = C(1.0 / (s->w[a] * s->scale));
    }
    k.inv_den = 1.0 / s->den;
    for (int p = 0; p < s->P; ++p) {
        const int a = s->R + p;
        const double x = s->ex[a], y = s->ey[a];
        k.pex[p] = C(x);
        k.pey[p] = C(y);
        k.pexx[p] = C(x * x);
        k.pexy2[p] = C(2 * x * y);
        k.peyy[p] = C(y * y);
        k.pge[p] = C(s->c * s->g * x);
        k.pomw[p] = C(omega * s->w[a]);
        const double ws = s->w[a] * s->scale;
        k.hw[p] = C(ws);
        k.hwx[p] = C(ws * x);
        k.hwy[p] = C(ws * y);
        k.hwxx[p] = C(ws * x * x);
        k.hwxy[p] = C(ws * x * y);
        k.hwyy[p] = C(ws * y * y);
    }
    k.hw_rest = C(s->R ? s->w[0] * s->scale : 0.0);
    k.fill_h = C(1.0 / s->scale);
    k.om_s = C(omega / s->scale);
    k.omw_rest = C(s->R ? omega * s->w[0] : 0.0);
    k.c = C(s->c);
    k.c2 = C(s->c * s->c);
    k.tau = C(s->tau);
    k.dt = C(s->dt);
    k.hdt = C(0.5 * s->dt);
    k.omega = C(omega);
    k.one_m_omega = C(1.0 - omega);
    k.gx = C(s->g);
    k.gy = C(0);
    k.two_tau = C(2 * s->tau);
    k.inv_2tau_dt = C(1.0 / (2 * s->tau + s->dt));
    k.half_tau = C(0.5 * s->tau);
    k.hdt_gx = k.hdt * k.gx;
    k.hdt_gy = k.hdt * k.gy;
    k.tgx = k.two_tau * k.gx;
    k.tgy = k.two_tau * k.gy;
    k.ttc2 = k.two_tau * k.c2;
    k.htc2 = k.half_tau * k.c2;
    k.tc = k.tau * k.c;
    k.cg = k.c * k.gx;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

__global__ void k_fill(double* p, int n, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Partial sums for the fp64 reductions: per block, sum of u_x and
// max |u_x - prev| (when prev is given).  Fixed shapes: deterministic.
__global__ void __launch_bounds__(lbm::kReduceThreads)
k_reduce_partial(const double* __restrict__ ux, const double* __restrict__ prev, int n,
                 double* __restrict__ partial) {
    __shared__ double ssum[lbm::kReduceThreads / 32], smax[lbm::kReduceThreads / 32];
    double s = 0.0, m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double u = ux[i];
        s += u;
        if (prev) m = fmax(m, fabs(u - prev[i]));
        if (u != u) m = u;   // propagate NaN into the convergence test
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        const double mo = __shfl_down_sync(0xffffffffu, m, o);
        m = (mo != mo) ? mo : fmax(m, mo);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { ssum[wid] = s; smax[wid] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = 0.0;
        for (int k = 0; k < lbm::kReduceThreads / 32; ++k) {
            ts += ssum[k];
            tm = (smax[k] != smax[k]) ? smax[k] : fmax(tm, smax[k]);
        }
        partial[2 * blockIdx.x] = ts;
        partial[2 * blockIdx.x + 1] = tm;
    }
}

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < int(blockDim.x >> 5); ++k) t += sh[k];
    return t;   // valid in thread 0
}

// Final reduction (one block of 256): mean u_x, max |du|, slip velocity
// (Eq. defSlip, quadratic wall extrapolation, centre interpolation) and the
// normalised mass flow (Eq. pf.1).
__global__ void __launch_bounds__(256)
k_reduce_final(const double* __restrict__ partial, int nblk, const double* __restrict__ ux,
               int Nx, int Ny, double tau, double g, double Kn, double* __restrict__ res) {
    __shared__ double sh[32];
    __shared__ double rows[10];
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        s += partial[2 * i];
        const double mi = partial[2 * i + 1];
        m = (mi != mi) ? mi : fmax(m, mi);
    }
    const double tot = block_sum(s, sh);
    // max over threads
    for (int o = 16; o > 0; o >>= 1) {
        const double mo = __shfl_down_sync(0xffffffffu, m, o);
        m = (mo != mo) ? mo : fmax(m, mo);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    double mx = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < int(blockDim.x >> 5); ++k) mx = (sh[k] != sh[k]) ? sh[k] : fmax(mx, sh[k]);
    __syncthreads();
    // row means of u_x for the slip velocity
    const int m2 = Ny / 2;
    int rlist[10] = {0, 1, 2, Ny - 1, Ny - 2, Ny - 3, m2 - 2, m2 - 1, m2, m2 + 1};
    if (Ny & 1) rlist[6] = rlist[7] = rlist[8] = rlist[9] = (Ny - 1) / 2;
    const bool slip_ok = Ny >= 4;
    for (int r = 0; r < 10; ++r) {
        double v = 0.0;
        if (slip_ok)
            for (int x = threadIdx.x; x < Nx; x += blockDim.x) v += ux[(long long)rlist[r] * Nx + x];
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) rows[r] = t / Nx;
    }
    if (threadIdx.x == 0) {
        const double mean = tot / ((double)Nx * Ny);
        res[0] = mean;
        res[1] = mx;
        double us = nan("");
        if (slip_ok) {
            const double bot = (15.0 * rows[0] - 10.0 * rows[1] + 3.0 * rows[2]) / 8.0;
            const double top = (15.0 * rows[3] - 10.0 * rows[4] + 3.0 * rows[5]) / 8.0;
            const double uc = (Ny & 1) ? rows[8]
                                       : (9.0 * (rows[7] + rows[8]) - (rows[6] + rows[9])) / 16.0;
            us = 0.5 * (bot + top) / uc;
        }
        res[2] = us;
        res[3] = g != 0.0 ? 2.0 * tau * mean / (g * Kn) : nan("");
    }
}

template <typename C>
void set_plane_pointers(const lbm_solver* s, KParams<C>& k, const void* src, void* dst) {
    const ptrdiff_t plane = ptrdiff_t(s->Nx) * s->Ny;
    const ptrdiff_t es = ptrdiff_t(s->elem);
    for (int a = 0; a < s->V; ++a) {
        k.srcf[a] = static_cast<const char*>(src) + (a * plane - k.off[a]) * es;
        k.dstp[a] = static_cast<char*>(dst) + a * plane * es;
    }
}

// Knudsen-layer diagnostic (Eq. uNS, uNEQ), one block: x-averaged u_x per row,
// u(0) as for the slip velocity, <u> over all nodes, then
// out[y] = u(y) - u(0) (1 - 3 (1 - <u>/u(0)) (2 z_y)^2), z_y = (y + 1/2)/Ny - 1/2.
__global__ void __launch_bounds__(256)
k_knudsen_layer(const double* __restrict__ ux, int Nx, int Ny, double* __restrict__ out) {
    __shared__ double sh[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int y = warp; y < Ny; y += 8) {
        double v = 0.0;
        for (int x = lane; x < Nx; x += 32) v += ux[(long long)y * Nx + x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[y] = v / Nx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mean = 0.0;
        for (int y = 0; y < Ny; ++y) mean += out[y];
        mean /= Ny;
        const int m = Ny / 2;
        const double uc = (Ny & 1) ? out[(Ny - 1) / 2]
                                   : (9.0 * (out[m - 1] + out[m]) - (out[m - 2] + out[m + 1])) / 16.0;
        sh[0] = uc;
        sh[1] = 3.0 * (1.0 - mean / uc);
    }
    __syncthreads();
    const double uc = sh[0], a = sh[1];
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) {
        const double z2 = 2.0 * ((y + 0.5) / Ny - 0.5);
        out[y] -= uc * (1.0 - a * z2 * z2);
    }
}

int launch_step(lbm_solver* s, int emit) {
    const void* src = static_cast<const char*>(s->b.f[s->cur]);
    void* dst = s->b.f[1 - s->cur];
    set_plane_pointers(s, s->k64, src, dst);
    set_plane_pointers(s, s->k32, src, dst);
    cudaError_t e;
    if (s->precision == LBM_FP64) {
        s->k64.emit = emit;
        e = lbm::launch_step_fp64(s->k64, s->N, src, dst, s->b, s->stream);
    } else if (s->precision == LBM_FP32) {
        s->k32.emit = emit;
        e = lbm::launch_step_fp32(s->k32, s->N, src, dst, s->b, s->stream);
    } else {
        s->k32.emit = emit;
        s->k32.seed = unsigned(s->steps + 1);
        e = lbm::launch_step_fp16(s->k32, s->N, s->precision == LBM_BF16, src, dst, s->b,
                                  s->stream);
    }
    if (e != cudaSuccess) return cuda_status(e);
    s->cur = 1 - s->cur;
    s->steps += 1;
    return LBM_OK;
}

int launch_init(lbm_solver* s, const double* rho_dev) {
    s->cur = 0;
    s->steps = 0;
    cudaError_t e = cudaMemsetAsync(s->b.status, 0, sizeof(unsigned), s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (is16(s->precision) && s->scale != 1.0 / 64.0) {
        s->scale = 1.0 / 64.0;
        lbm::fill_params(*s, s->k32);
    }
    if (s->precision == LBM_FP64) {
        s->k64.emit = 1;
        e = lbm::launch_init_fp64(s->k64, s->N, rho_dev, s->b.f[0], s->b, s->stream);
    } else if (s->precision == LBM_FP32) {
        s->k32.emit = 1;
        e = lbm::launch_init_fp32(s->k32, s->N, rho_dev, s->b.f[0], s->b, s->stream);
    } else {
        s->k32.emit = 1;
        s->k32.seed = 0u;
        e = lbm::launch_init_fp16(s->k32, s->N, s->precision == LBM_BF16, rho_dev, s->b.f[0],
                                  s->b, s->stream);
    }
    return cuda_status(e);
}

int reduce(lbm_solver* s, bool with_prev, double out[4]) {
    const int n = s->Nx * s->Ny;
    k_reduce_partial<<<lbm::kReduceBlocks, lbm::kReduceThreads, 0, s->stream>>>(
        s->b.ux, with_prev ? s->b.prev_ux : nullptr, n, s->b.partial);
    k_reduce_final<<<1, 256, 0, s->stream>>>(s->b.partial, lbm::kReduceBlocks, s->b.ux, s->Nx,
                                             s->Ny, s->tau, s->g, s->Kn, s->b.results);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, s->b.results, 4 * sizeof(double),
                                              cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

int read_status(lbm_solver* s) {
    unsigned st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, s->b.status, sizeof(st), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return st ? LBM_ENONFINITE : LBM_OK;
}

// 16-bit storage: make max |h| over the state lie in (1/2, 1] by a power-of-2
// change of S (exact up to the format's subnormal range).  Synchronises.
int refresh_scale(lbm_solver* s) {
    if (!is16(s->precision)) return LBM_OK;
    const long long n = (long long)s->V * s->Nx * s->Ny;
    float* out = reinterpret_cast<float*>(s->b.results + 6);
    const bool bf = s->precision == LBM_BF16;
    cudaError_t e = lbm::launch_absmax_fp16(s->b.f[s->cur], n, bf, out, s->stream);
    float m = 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, out, sizeof(m), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (!(m > 0.f) || !std::isfinite(m)) return LBM_OK;
    const double target = std::ldexp(1.0, int(std::ceil(std::log2(double(m) * s->scale))));
    const double ns = std::max(target, std::ldexp(1.0, -40));
    if (ns == s->scale) return LBM_OK;
    e = lbm::launch_rescale_fp16(s->b.f[s->cur], n, bf, float(s->scale / ns), s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->scale = ns;
    lbm::fill_params(*s, s->k32);
    return LBM_OK;
}

bool resident_on(const lbm_solver* s) {
    return s->resident && s->cl.ctas > 0 &&
           (s->precision == LBM_FP64 || s->precision == LBM_FP32);
}

// K >= 1 steps on the resident cluster kernel, at most kClusterMaxK per launch;
// the last step writes the moments, and with emit_prev the step before it
// writes u_x to prev_ux (the final launch keeps >= 2 steps for that).
int resident_steps(lbm_solver* s, long K, bool emit_prev) {
    while (K > 0) {
        const long n = K <= lbm::kClusterMaxK ? K : std::min(lbm::kClusterMaxK, K - 2);
        const int next = int((s->cur + n) & 1);
        const bool prev = emit_prev && n == K;
        const cudaError_t e =
            s->precision == LBM_FP64
                ? lbm::launch_chunk_cluster(s->k64, s->cl, s->b.f[s->cur], s->b.f[next], s->b,
                                            int(n), prev, s->stream)
                : lbm::launch_chunk_cluster(s->k32, s->cl, s->b.f[s->cur], s->b.f[next], s->b,
                                            int(n), prev, s->stream);
        if (e != cudaSuccess) return cuda_status(e);
        s->cur = next;
        s->steps += n;
        K -= n;
    }
    return LBM_OK;
}

// Enqueue one convergence chunk: K-1 steps (the last emitting moments), the
// copy u_x -> prev, one more step, and the fp64 reductions into b.results.
// Resident channels do the K steps in one launch that writes prev itself.
int enqueue_chunk(lbm_solver* s, long K) {
    if (resident_on(s) && K >= 2) {
        const int rc = resident_steps(s, K, true);
        if (rc) return rc;
    } else {
        for (long i = 0; i < K - 1; ++i) {
            const int rc = launch_step(s, i == K - 2);
            if (rc) return rc;
        }
        cudaError_t e = cudaMemcpyAsync(s->b.prev_ux, s->b.ux, size_t(s->Nx) * s->Ny * 8,
                                        cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_status(e);
        const int rc = launch_step(s, true);
        if (rc) return rc;
    }
    const int n = s->Nx * s->Ny;
    k_reduce_partial<<<lbm::kReduceBlocks, lbm::kReduceThreads, 0, s->stream>>>(
        s->b.ux, s->b.prev_ux, n, s->b.partial);
    k_reduce_final<<<1, 256, 0, s->stream>>>(s->b.partial, lbm::kReduceBlocks, s->b.ux, s->Nx,
                                             s->Ny, s->tau, s->g, s->Kn, s->b.results);
    return cuda_status(cudaGetLastError());
}

// One chunk replayed from a CUDA graph (captured on first use for the current
// lattice parity); the step counter and lattice index advance as if launched.
int graph_chunk(lbm_solver* s, long K) {
    const int par = s->cur;
    if (!s->chunk_exec[par] || s->chunk_K[par] != K) {
        if (s->chunk_exec[par]) {
            cudaGraphExecDestroy(s->chunk_exec[par]);
            s->chunk_exec[par] = nullptr;
        }
        const int cur0 = s->cur;
        const long steps0 = s->steps;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e);
        const int rc = enqueue_chunk(s, K);
        e = cudaStreamEndCapture(s->stream, &g);
        s->cur = cur0;
        s->steps = steps0;
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : cuda_status(e);
        }
        e = cudaGraphInstantiate(&s->chunk_exec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_status(e);
        s->chunk_K[par] = K;
    }
    const cudaError_t e = cudaGraphLaunch(s->chunk_exec[par], s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->cur = int((par + K) & 1);
    s->steps += K;
    return LBM_OK;
}

int create_common(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn, double force,
                  int precision, void* stream, void* workspace, size_t bytes, bool own,
                  lbm_solver** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_solver* s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ENOMEM;
    int rc = lbm::prepare_spec(dvm, order, Nx, Ny, Kn, force, precision, *s);
    if (rc) { delete s; return rc; }
    s->stream = static_cast<cudaStream_t>(stream);
    const Layout L = layout(s->V, size_t(Nx) * Ny, s->elem);
    if (own) {
        cudaError_t e = cudaMalloc(&s->ws, L.total);
        if (e != cudaSuccess) { delete s; return LBM_ENOMEM; }
        s->owns = true;
    } else {
        if (!workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
            delete s;
            return workspace && bytes < L.total ? LBM_ENOMEM : LBM_EINVAL;
        }
        s->ws = workspace;
    }
    s->ws_bytes = L.total;
    char* base = static_cast<char*>(s->ws);
    s->b.f[0] = base + L.f0;
    s->b.f[1] = base + L.f1;
    s->b.rho = reinterpret_cast<double*>(base + L.rho);
    s->b.ux = reinterpret_cast<double*>(base + L.ux);
    s->b.uy = reinterpret_cast<double*>(base + L.uy);
    s->b.prev_ux = reinterpret_cast<double*>(base + L.prev);
    s->b.partial = reinterpret_cast<double*>(base + L.partial);
    s->b.results = reinterpret_cast<double*>(base + L.results);
    s->b.status = reinterpret_cast<unsigned*>(base + L.status);
    lbm::fill_params(*s, s->k64);
    lbm::fill_params(*s, s->k32);
    if (precision == LBM_FP64 || precision == LBM_FP32) {
        const int LP = lbm::warp_path_lanes(s->P, (long long)Nx * Ny);
        if (LP && precision == LBM_FP64) lbm::plan_cluster(s->k64, s->N, LP, s->cl);
        if (LP && precision == LBM_FP32) lbm::plan_cluster(s->k32, s->N, LP, s->cl);
    }
    *out = s;
    return LBM_OK;
}

}  // namespace

namespace lbm {

int prepare_spec(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn, double force,
                 int precision, SolveSpec& s) {
    if (!valid_precision(precision)) return LBM_EINVAL;
    if (Nx < 1 || Ny < 1 || !(Kn > 0) || !std::isfinite(Kn) || !std::isfinite(force))
        return LBM_EINVAL;
    if ((long long)Nx * Ny > (long long)0x7fffffff) return LBM_EINVAL;
    int rc = canonicalize(dvm, s.ex, s.ey, s.w, s.perm, s.R, s.P, s.set_id);
    if (rc) return rc;
    int Q = -1;
    lbm_dvm_quadrature_order(dvm, &Q);
    if (order < 2 || order > 4 || Q < 5 || Q < 2 * order - 1) return LBM_EDEGREE;
    s.V = dvm->V;
    s.maxey = s.maxex = 0;
    for (int a = 0; a < s.V; ++a) {
        s.maxey = std::max(s.maxey, std::abs(s.ey[a]));
        s.maxex = std::max(s.maxex, std::abs(s.ex[a]));
    }
    if (Ny < s.maxey || s.maxey == 0) return LBM_EINVAL;
    s.precision = precision;
    s.N = order;
    s.Nx = Nx;
    s.Ny = Ny;
    s.c = dvm->c;
    s.Kn = Kn;
    s.tau = std::sqrt(2.0 / M_PI) * Kn;    // Eq. nm.13
    s.dt = (1.0 / Ny) / dvm->c;            // dx = l0 / Ny, one hop per step
    s.g = force;
    s.den = 0.0;
    for (int a = 0; a < s.V; ++a)
        if (s.ey[a] > 0) s.den += s.ey[a] * s.w[a];
    s.elem = elem_bytes(precision);
    s.scale = 1.0 / 64.0;
    return LBM_OK;
}

template <typename C>
void fill_params(const SolveSpec& s, KParams<C>& k) { fill_params_impl(&s, k); }
template void fill_params<float>(const SolveSpec&, KParams<float>&);
template void fill_params<double>(const SolveSpec&, KParams<double>&);

}  // namespace lbm

extern "C" {

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_EDEGREE: return "quadrature order too low for the Hermite order";
        case LBM_ENOMEM: return "out of device memory or workspace too small";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_ENONFINITE: return "non-finite or non-positive density";
        case LBM_ETIMEOUT: return "bounded device wait timed out";
        case LBM_ENOTCONV: return "not converged within max_steps";
        case LBM_ENOTSUP: return "not supported";
        default: return "unknown error";
    }
}

int lbm_workspace_bytes(const lbm_dvm* dvm, int Nx, int Ny, int precision, size_t* bytes) {
    if (!dvm || !bytes || Nx < 1 || Ny < 1 || dvm->V < 1 || dvm->V > LBM_MAX_V) return LBM_EINVAL;
    if (!valid_precision(precision)) return LBM_EINVAL;
    *bytes = layout(dvm->V, size_t(Nx) * Ny, elem_bytes(precision)).total;
    return LBM_OK;
}

int lbm_create(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn, double force,
               int precision, void* stream, lbm_solver** out) {
    return create_common(dvm, order, Nx, Ny, Kn, force, precision, stream, nullptr, 0, true, out);
}

int lbm_create_in(const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn, double force,
                  int precision, void* stream, void* workspace, size_t bytes,
                  lbm_solver** out) {
    return create_common(dvm, order, Nx, Ny, Kn, force, precision, stream, workspace, bytes,
                         false, out);
}

void lbm_destroy(lbm_solver* s) {
    if (!s) return;
    for (auto& g : s->chunk_exec)
        if (g) cudaGraphExecDestroy(g);
    if (s->owns && s->ws) {
        cudaStreamSynchronize(s->stream);
        cudaFree(s->ws);
    }
    delete s;
}

int lbm_init(lbm_solver* s, const double* rho_host) {
    if (!s) return LBM_EINVAL;
    const int n = s->Nx * s->Ny;
    cudaError_t e;
    if (rho_host)
        e = cudaMemcpyAsync(s->b.prev_ux, rho_host, size_t(n) * 8, cudaMemcpyHostToDevice, s->stream);
    else {
        k_fill<<<(n + 255) / 256, 256, 0, s->stream>>>(s->b.prev_ux, n, 1.0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_status(e);
    return launch_init(s, s->b.prev_ux);
}

int lbm_init_device(lbm_solver* s, const double* rho_device) {
    if (!s || !rho_device) return LBM_EINVAL;
    return launch_init(s, rho_device);
}

int lbm_step(lbm_solver* s, long nsteps) {
    if (!s || nsteps < 0) return LBM_EINVAL;
    if (resident_on(s) && nsteps >= 2) return resident_steps(s, nsteps, false);
    for (long i = 0; i < nsteps; ++i) {
        const int rc = launch_step(s, i == nsteps - 1);
        if (rc) return rc;
    }
    return LBM_OK;
}

__global__ void k_scale3(double* a, double* b, double* c, long long n, double f) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        a[i] *= f;
        b[i] *= f;
        c[i] *= f;
    }
}

int lbm_average(lbm_solver* s, long nsteps, long every) {
    if (!s || every < 1 || nsteps < every) return LBM_EINVAL;
    const long long n = (long long)s->Nx * s->Ny;
    cudaError_t e = cudaSuccess;
    for (double* f : {s->b.rho, s->b.ux, s->b.uy})
        if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, size_t(n) * 8, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    long count = 0;
    for (long i = 1; i <= nsteps; ++i) {
        const bool sample = i % every == 0;
        const int rc = launch_step(s, sample ? 2 : 0);
        if (rc) return rc;
        count += sample;
    }
    const int blocks = int(std::min<long long>((n + 255) / 256, 4 * 152));
    k_scale3<<<blocks, 256, 0, s->stream>>>(s->b.rho, s->b.ux, s->b.uy, n, 1.0 / double(count));
    return cuda_status(cudaGetLastError());
}

int lbm_run_to_steady(lbm_solver* s, double tol, long max_steps, long check_every,
                      long* steps_done, double* last_du) {
    if (!s || !(tol > 0) || max_steps < 0 || check_every < 2) return LBM_EINVAL;
    double du = HUGE_VAL;
    int rc = LBM_ENOTCONV;
    // on a capturable stream, fp32/fp64 chunks replay a CUDA graph
    const bool graphs = s->stream != nullptr && !is16(s->precision);
    while (s->steps < max_steps) {
        const long n = std::min(check_every, max_steps - s->steps);
        double r[4];
        if (graphs) {
            if ((rc = graph_chunk(s, n))) break;
            cudaError_t e = cudaMemcpyAsync(r, s->b.results, 4 * sizeof(double),
                                            cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) { rc = cuda_status(e); break; }
        } else {
            if ((rc = enqueue_chunk(s, n))) break;
            cudaError_t e = cudaMemcpyAsync(r, s->b.results, 4 * sizeof(double),
                                            cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) { rc = cuda_status(e); break; }
        }
        du = r[1];
        if ((rc = read_status(s))) break;
        if ((rc = refresh_scale(s))) break;
        rc = LBM_ENOTCONV;
        if (du < tol) { rc = LBM_OK; break; }
    }
    if (steps_done) *steps_done = s->steps;
    if (last_du) *last_du = du;
    return rc;
}

int lbm_set_resident(lbm_solver* s, int enable) {
    if (!s || (enable != 0 && enable != 1)) return LBM_EINVAL;
    if (s->resident != bool(enable)) {
        for (int i = 0; i < 2; ++i) {
            if (s->chunk_exec[i]) cudaGraphExecDestroy(s->chunk_exec[i]);
            s->chunk_exec[i] = nullptr;
            s->chunk_K[i] = 0;
        }
    }
    s->resident = bool(enable);
    return LBM_OK;
}

int lbm_resident_ctas(lbm_solver* s, int* ctas) {
    if (!s || !ctas) return LBM_EINVAL;
    *ctas = resident_on(s) ? s->cl.ctas : 0;
    return LBM_OK;
}

int lbm_moments(lbm_solver* s, double* rho, double* ux, double* uy) {
    if (!s) return LBM_EINVAL;
    const size_t n = size_t(s->Nx) * s->Ny * 8;
    cudaError_t e = cudaSuccess;
    if (rho && e == cudaSuccess) e = cudaMemcpyAsync(rho, s->b.rho, n, cudaMemcpyDeviceToHost, s->stream);
    if (ux && e == cudaSuccess) e = cudaMemcpyAsync(ux, s->b.ux, n, cudaMemcpyDeviceToHost, s->stream);
    if (uy && e == cudaSuccess) e = cudaMemcpyAsync(uy, s->b.uy, n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return read_status(s);
}

int lbm_mass_flow(lbm_solver* s, double* mdot, double* mean_ux) {
    if (!s) return LBM_EINVAL;
    double r[4];
    int rc = reduce(s, false, r);
    if (rc) return rc;
    if (mdot) *mdot = r[3];
    if (mean_ux) *mean_ux = r[0];
    return read_status(s);
}

int lbm_slip_velocity(lbm_solver* s, double* us) {
    if (!s || !us) return LBM_EINVAL;
    if (s->Ny < 4) return LBM_EINVAL;
    double r[4];
    int rc = reduce(s, false, r);
    if (rc) return rc;
    *us = r[2];
    return read_status(s);
}

int lbm_knudsen_layer(lbm_solver* s, double* uneq) {
    if (!s || !uneq || s->Ny < 4) return LBM_EINVAL;
    k_knudsen_layer<<<1, 256, 0, s->stream>>>(s->b.ux, s->Nx, s->Ny, s->b.prev_ux);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(uneq, s->b.prev_ux, size_t(s->Ny) * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return read_status(s);
}

int lbm_status(lbm_solver* s) {
    if (!s) return LBM_EINVAL;
    return read_status(s);
}

int lbm_steps_done(lbm_solver* s, long* steps) {
    if (!s || !steps) return LBM_EINVAL;
    *steps = s->steps;
    return LBM_OK;
}

int lbm_populations(lbm_solver* s, double* f_host) {
    if (!s || !f_host) return LBM_EINVAL;
    const size_t n = size_t(s->Nx) * s->Ny;
    std::vector<char> raw(size_t(s->V) * n * s->elem);
    cudaError_t e = cudaMemcpyAsync(raw.data(), s->b.f[s->cur], raw.size(), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int a = 0; a < s->V; ++a) {
        double* dst = f_host + size_t(s->perm[a]) * n;
        for (size_t i = 0; i < n; ++i) {
            double d;
            if (s->precision == LBM_FP64)
                d = reinterpret_cast<const double*>(raw.data())[a * n + i];
            else if (s->precision == LBM_FP32)
                d = double(reinterpret_cast<const float*>(raw.data())[a * n + i]);
            else if (s->precision == LBM_FP16)
                d = double(__half2float(reinterpret_cast<const __half*>(raw.data())[a * n + i])) *
                    double(s->k32.sw[a]);
            else
                d = double(__bfloat162float(
                        reinterpret_cast<const __nv_bfloat16*>(raw.data())[a * n + i])) *
                    double(s->k32.sw[a]);
            dst[i] = s->w[a] + d;
        }
    }
    return LBM_OK;
}

int lbm_state_bytes(lbm_solver* s, size_t* bytes) {
    if (!s || !bytes) return LBM_EINVAL;
    const size_t n = size_t(s->Nx) * s->Ny;
    *bytes = sizeof(StateHeader) + size_t(s->V) * n * s->elem + 3 * n * 8;
    return LBM_OK;
}

int lbm_get_state(lbm_solver* s, void* host, size_t bytes) {
    size_t need = 0;
    if (!host || lbm_state_bytes(s, &need) || bytes < need) return LBM_EINVAL;
    const size_t n = size_t(s->Nx) * s->Ny;
    StateHeader h{kStateMagic, s->precision, s->V, s->Nx, s->Ny, s->N, s->steps, s->scale};
    std::memcpy(host, &h, sizeof(h));
    char* p = static_cast<char*>(host) + sizeof(h);
    const size_t fb = size_t(s->V) * n * s->elem;
    cudaError_t e = cudaMemcpyAsync(p, s->b.f[s->cur], fb, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + fb, s->b.rho, n * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + fb + n * 8, s->b.ux, n * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + fb + 2 * n * 8, s->b.uy, n * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

int lbm_set_state(lbm_solver* s, const void* host, size_t bytes) {
    size_t need = 0;
    if (!host || lbm_state_bytes(s, &need) || bytes < need) return LBM_EINVAL;
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != kStateMagic || h.precision != s->precision || h.V != s->V || h.Nx != s->Nx ||
        h.Ny != s->Ny || h.N != s->N || h.steps < 0)
        return LBM_EINVAL;
    const size_t n = size_t(s->Nx) * s->Ny;
    const char* p = static_cast<const char*>(host) + sizeof(h);
    const size_t fb = size_t(s->V) * n * s->elem;
    s->cur = 0;
    cudaError_t e = cudaMemcpyAsync(s->b.f[0], p, fb, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->b.rho, p + fb, n * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->b.ux, p + fb + n * 8, n * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->b.uy, p + fb + 2 * n * 8, n * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->b.status, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->steps = h.steps;
    if (is16(s->precision)) {
        s->scale = h.scale;
        lbm::fill_params(*s, s->k32);
    }
    return LBM_OK;
}

}  // extern "C"
