// Engine kernels with 16-bit population storage (IEEE half, bfloat16).
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_step_fp16(int set_id, int N, bool bf16, const EngineLaunch& L, cudaStream_t st) {
    return bf16 ? engine_step_t<__nv_bfloat16>(set_id, N, L, st)
                : engine_step_t<__half>(set_id, N, L, st);
}

int engine_occupancy_fp16(int set_id, int N, bool bf16) {
    return bf16 ? engine_occupancy_t<__nv_bfloat16>(set_id, N) : engine_occupancy_t<__half>(set_id, N);
}

}  // namespace lbm
