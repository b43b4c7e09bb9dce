// lbm_observables_noalloc: the fp64 observables reduction (mean u_x, mass
// flow, slip velocity) for callers that cannot allocate device memory.
//
// Its scratch (one partial sum per block) lives in a file-scope __device__
// array instead of memory from cudaMalloc or a workspace.  The array exists
// once per device that loads this library and is held until the process
// exits.  Host code only ever sees a host-side stand-in for the array's name,
// so the device address is looked up with cudaGetSymbolAddress, with the
// device current, and handed to the kernels.  The address belongs to the
// device's current context: it is looked up once per device and again
// whenever the context changes (after a cudaDeviceReset the module is loaded
// anew and the array may move).
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                    // nodes per thread
constexpr int kMaxPartials = 4096;            // blocks, one partial each
constexpr long long kMaxNodes = (long long)kMaxPartials * kThreads * kItems;   // 16,777,216
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: kMaxPartials doubles (32 KiB).
static __device__ __align__(256) double g_noalloc_partial[kMaxPartials];

// Per device: the unique id of the context the address was looked up in
// (a context handle can be reused after a reset; its id is not), and the
// address.
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points
// (the library does not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
void* driver_fn(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return p;
}

// Unique id of the calling thread's current context (0: none).
int current_context_id(unsigned long long* id) {
    static const CtxGetCurrentFn get_ctx =
        reinterpret_cast<CtxGetCurrentFn>(driver_fn("cuCtxGetCurrent"));
    static const CtxGetIdFn get_id = reinterpret_cast<CtxGetIdFn>(driver_fn("cuCtxGetId"));
    if (!get_ctx || !get_id) return LBM_ECUDA;
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return LBM_ECUDA;
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return LBM_ECUDA;
    return LBM_OK;
}

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
// the first call per device and again when the device's context has changed.
int scratch_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return LBM_ECUDA;
    if (dev >= kMaxDevices) return LBM_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_scratch[dev];
    unsigned long long id = 0;
    if (current_context_id(&id)) return LBM_ECUDA;
    if (id == 0 || id != slot.ctx_id || !slot.ptr) {
        // the lookup also creates the device's primary context if there is none yet
        void* addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_noalloc_partial) != cudaSuccess || !addr)
            return LBM_ECUDA;
        if (current_context_id(&id) || id == 0) return LBM_ECUDA;
        slot.ctx_id = id;
        slot.ptr = static_cast<double*>(addr);
    }
    *out = slot.ptr;
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
    // an error already pending on this thread belongs to earlier work: leave
    // it for its owner (cudaPeekAtLastError does not clear it) and refuse
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
    double* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    const int nblk = int((n + (long long)kThreads * kItems - 1) / ((long long)kThreads * kItems));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double tau = std::sqrt(2.0 / M_PI) * Kn;   // Eq. nm.13, as in lbm_create
    k_noalloc_partial<<<nblk, kThreads, 0, st>>>(ux_device, n, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();   // this call's own launch error: report it and clear it
        return LBM_ECUDA;
    }
    k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, nblk, ux_device, Nx, Ny, tau, force, Kn,
                                            out_device);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    return LBM_OK;
}
