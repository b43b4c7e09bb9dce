// lbm_observables_noalloc: the fp64 observables reduction (mean u_x, mass
// flow, slip velocity) for callers that cannot allocate device memory.
//
// Its scratch (one partial sum per block) lives in a file-scope __device__
// array instead of memory from cudaMalloc or a workspace.  The array exists
// once per device that loads this library and is held until the process
// exits.  Host code only ever sees a host-side stand-in for the array's name,
// so the device address is looked up with cudaGetSymbolAddress, once per
// device, with that device current, and handed to the kernels.
#include <atomic>
#include <cmath>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                    // nodes per thread
constexpr int kMaxPartials = 4096;            // blocks, one partial each
constexpr long long kMaxNodes = (long long)kMaxPartials * kThreads * kItems;   // 16,777,216
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: kMaxPartials doubles (32 KiB).
static __device__ __align__(256) double g_noalloc_partial[kMaxPartials];

std::atomic<double*> g_scratch[kMaxDevices];

__device__ double block_sum_na(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    return t;   // valid in thread 0
}

// One partial sum of u_x per block: block b covers nodes
// [b * kThreads * kItems, (b + 1) * kThreads * kItems).
__global__ void __launch_bounds__(kThreads)
k_noalloc_partial(const double* __restrict__ ux, long long n, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    const long long base = (long long)blockIdx.x * kThreads * kItems;
    double s = 0.0;
    for (int i = 0; i < kItems; ++i) {
        const long long j = base + (long long)i * kThreads + threadIdx.x;
        if (j < n) s += ux[j];
    }
    const double t = block_sum_na(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Combine the partials and evaluate the observables (same definitions as
// lbm_mass_flow and lbm_slip_velocity): out = {mean u_x, mdot, u_s}.
__global__ void __launch_bounds__(kThreads)
k_noalloc_final(const double* __restrict__ partial, int nblk, const double* __restrict__ ux,
                int Nx, int Ny, double tau, double g, double Kn, double* __restrict__ out) {
    __shared__ double sh[kThreads / 32];
    __shared__ double rows[10];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) s += partial[i];
    const double tot = block_sum_na(s, sh);
    const int m2 = Ny / 2;
    int rlist[10] = {0, 1, 2, Ny - 1, Ny - 2, Ny - 3, m2 - 2, m2 - 1, m2, m2 + 1};
    if (Ny & 1) rlist[6] = rlist[7] = rlist[8] = rlist[9] = (Ny - 1) / 2;
    for (int r = 0; r < 10; ++r) {
        double v = 0.0;
        for (int x = threadIdx.x; x < Nx; x += kThreads) v += ux[(long long)rlist[r] * Nx + x];
        const double t = block_sum_na(v, sh);
        if (threadIdx.x == 0) rows[r] = t / Nx;
    }
    if (threadIdx.x == 0) {
        const double mean = tot / ((double)Nx * Ny);
        const double bot = (15.0 * rows[0] - 10.0 * rows[1] + 3.0 * rows[2]) / 8.0;
        const double top = (15.0 * rows[3] - 10.0 * rows[4] + 3.0 * rows[5]) / 8.0;
        const double uc = (Ny & 1) ? rows[8] : (9.0 * (rows[7] + rows[8]) - (rows[6] + rows[9])) / 16.0;
        out[0] = mean;
        out[1] = g != 0.0 ? 2.0 * tau * mean / (g * Kn) : nan("");
        out[2] = 0.5 * (bot + top) / uc;
    }
}

// Device address of the scratch array on the current device, looked up on
// the first call per device.
int scratch_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return LBM_ECUDA;
    if (dev >= kMaxDevices) return LBM_ENOTSUP;
    double* p = g_scratch[dev].load(std::memory_order_acquire);
    if (!p) {
        void* addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_noalloc_partial) != cudaSuccess || !addr)
            return LBM_ECUDA;
        p = static_cast<double*>(addr);
        g_scratch[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_observables_noalloc(const double* ux_device, int Nx, int Ny, double Kn,
                                       double force, double* out_device, void* stream) {
    if (!ux_device || !out_device || Nx < 1 || Ny < 4 || !(Kn > 0) || !std::isfinite(Kn) ||
        !std::isfinite(force))
        return LBM_EINVAL;
    const long long n = (long long)Nx * Ny;
    if (n > kMaxNodes) return LBM_EINVAL;
    double* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    const int nblk = int((n + (long long)kThreads * kItems - 1) / ((long long)kThreads * kItems));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double tau = std::sqrt(2.0 / M_PI) * Kn;   // Eq. nm.13, as in lbm_create
    k_noalloc_partial<<<nblk, kThreads, 0, st>>>(ux_device, n, scratch);
    k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, nblk, ux_device, Nx, Ny, tau, force, Kn,
                                            out_device);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
