// fp32 instantiations of the stream-collide kernels: deviations fbar - w
// stored and computed in float; wall fluxes and moments handed out in double.
#include "lbm_kernels.cuh"

namespace lbm {

cudaError_t launch_step_fp32(const KParams<float>& k, int N, const void* src, void* dst,
                             const DevBufs& b, cudaStream_t st) {
    return launch_step_t<float, float>(k, N, src, dst, b, st);
}

cudaError_t launch_init_fp32(const KParams<float>& k, int N, const double* rho0, void* dst,
                             const DevBufs& b, cudaStream_t st) {
    return launch_init_t<float, float>(k, N, rho0, dst, b, st);
}

}  // namespace lbm
