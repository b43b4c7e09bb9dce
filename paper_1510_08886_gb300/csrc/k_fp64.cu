// fp64 instantiations of the stream-collide kernels: storage and arithmetic
// in double.
#include "lbm_kernels.cuh"

namespace lbm {

cudaError_t launch_step_fp64(const KParams<double>& k, int N, const void* src, void* dst,
                             const DevBufs& b, cudaStream_t st) {
    return launch_step_t<double, double>(k, N, src, dst, b, st);
}

cudaError_t launch_init_fp64(const KParams<double>& k, int N, const double* rho0, void* dst,
                             const DevBufs& b, cudaStream_t st) {
    return launch_init_t<double, double>(k, N, rho0, dst, b, st);
}

}  // namespace lbm
