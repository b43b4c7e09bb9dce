// bfloat16-storage instantiations of the stream-collide and init kernels
// (populations stored as h = (fbar - w) / (w S), arithmetic in fp32), in a
// translation unit of their own so that they compile in parallel with the
// IEEE-half ones.  Reached through launch_step_fp16 / launch_init_fp16.
#include "lbm_kernels.cuh"

namespace lbm {

cudaError_t launch_step_bf16_only(const KParams<float>& k, int N, const void* src, void* dst,
                                  const DevBufs& b, cudaStream_t st) {
    return launch_step_t<__nv_bfloat16, float>(k, N, src, dst, b, st);
}

cudaError_t launch_init_bf16_only(const KParams<float>& k, int N, const double* rho0, void* dst,
                                  const DevBufs& b, cudaStream_t st) {
    return launch_init_t<__nv_bfloat16, float>(k, N, rho0, dst, b, st);
}

}  // namespace lbm
