// Engine kernels with bfloat16 population storage.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_step_bf16(int set_id, int N, const EngineLaunch& L, cudaStream_t st) {
    return engine_step_t<__nv_bfloat16>(set_id, N, L, st);
}

int engine_occupancy_bf16(int set_id, int N) { return engine_occupancy_t<__nv_bfloat16>(set_id, N); }

}  // namespace lbm
