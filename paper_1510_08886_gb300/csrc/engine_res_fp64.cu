// Resident-chunk engine kernels, fp64 population storage and arithmetic.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_resident_fp64(int set_id, int N, const ResidentLaunch& L, cudaStream_t st) {
    return engine_resident_t<double>(set_id, N, L, st);
}

int engine_resident_attr_fp64(int set_id, int N, size_t smem) {
    return engine_resident_attr_t<double>(set_id, N, smem);
}

}  // namespace lbm
