// 16-bit storage instantiations of the stream-collide kernels: populations
// stored as h = (fbar - w) / (w S), arithmetic in fp32, wall fluxes and
// moments in fp64.  IEEE half here; bfloat16 in k_bf16.cu (its own
// translation unit, compiled in parallel), reached through the same two
// launchers.  Also the two state-wide helpers of the per-solve scale S: the
// max |h| reduction and the power-of-2 rescale.
#include "lbm_kernels.cuh"

namespace lbm {

// k_bf16.cu
cudaError_t launch_step_bf16_only(const KParams<float>& k, int N, const void* src, void* dst,
                                  const DevBufs& b, cudaStream_t st);
cudaError_t launch_init_bf16_only(const KParams<float>& k, int N, const double* rho0, void* dst,
                                  const DevBufs& b, cudaStream_t st);

cudaError_t launch_step_fp16(const KParams<float>& k, int N, bool bf16, const void* src, void* dst,
                             const DevBufs& b, cudaStream_t st) {
    return bf16 ? launch_step_bf16_only(k, N, src, dst, b, st)
                : launch_step_t<__half, float>(k, N, src, dst, b, st);
}

cudaError_t launch_init_fp16(const KParams<float>& k, int N, bool bf16, const double* rho0,
                             void* dst, const DevBufs& b, cudaStream_t st) {
    return bf16 ? launch_init_bf16_only(k, N, rho0, dst, b, st)
                : launch_init_t<__half, float>(k, N, rho0, dst, b, st);
}

template <typename S>
__global__ void __launch_bounds__(256) k_absmax(const S* __restrict__ f, long long n,
                                                float* __restrict__ out) {
    float m = 0.f;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        m = fmaxf(m, fabsf(Storage<S>::to_f(f[i])));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    // non-negative floats order like their bit patterns: atomicMax on the bits
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(m));
}

template <typename S>
__global__ void __launch_bounds__(256) k_rescale(S* __restrict__ f, long long n, float factor) {
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        f[i] = Storage<S>::from_f(Storage<S>::to_f(f[i]) * factor);
}

cudaError_t launch_absmax_fp16(const void* f, long long n, bool bf16, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (bf16)
        k_absmax<<<4 * 152, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(f), n, out);
    else
        k_absmax<<<4 * 152, 256, 0, st>>>(static_cast<const __half*>(f), n, out);
    return cudaGetLastError();
}

cudaError_t launch_rescale_fp16(void* f, long long n, bool bf16, float factor, cudaStream_t st) {
    if (bf16)
        k_rescale<<<4 * 152, 256, 0, st>>>(static_cast<__nv_bfloat16*>(f), n, factor);
    else
        k_rescale<<<4 * 152, 256, 0, st>>>(static_cast<__half*>(f), n, factor);
    return cudaGetLastError();
}

}  // namespace lbm
