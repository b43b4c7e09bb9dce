// Engine kernels with IEEE half population storage.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_step_half(int set_id, int N, const EngineLaunch& L, cudaStream_t st) {
    return engine_step_t<__half>(set_id, N, L, st);
}

int engine_occupancy_half(int set_id, int N) { return engine_occupancy_t<__half>(set_id, N); }

}  // namespace lbm
