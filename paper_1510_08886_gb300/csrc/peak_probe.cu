// lbm_fma_rate: the device's sustained FMA rate in fp64 or fp32, the
// denominator of the roofline of an arithmetic-bound step (the fp64 step on
// a part whose fp64 rate is far below its memory bandwidth's needs).
//
// Every thread runs kChains independent dependent chains a = a * b + c; the
// grid fills every SM several times over, so the FMA pipes, not latency,
// set the pace.  Timed with CUDA events on the caller's stream after one
// untimed launch; the best of three timed launches is reported.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* __restrict__ out, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int measure(int iters, cudaStream_t st, double* flops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ECUDA;
    const int blocks = sms * 8;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * kThreads) != cudaSuccess) return LBM_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = LBM_ECUDA;
    double best = 0.0;
    for (int r = 0; r < 4 && rc == LBM_OK; ++r) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<blocks, kThreads, 0, st>>>(out, iters, T(0.9999999), T(1e-7));
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = LBM_ECUDA;
            break;
        }
        const double f = 2.0 * double(blocks) * kThreads * kChains * double(iters) / (1e-3 * ms);
        if (r > 0) best = std::max(best, f);      // the first launch is a warm-up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc == LBM_OK && cudaGetLastError() != cudaSuccess) rc = LBM_ECUDA;
    *flops = best;
    return rc;
}

}  // namespace

extern "C" int lbm_fma_rate(int precision, void* stream, double* flops_per_s) {
    if (!flops_per_s || (precision != LBM_FP64 && precision != LBM_FP32)) return LBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return precision == LBM_FP64 ? measure<double>(20000, st, flops_per_s)
                                 : measure<float>(400000, st, flops_per_s);
}
