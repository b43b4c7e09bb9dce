// Resident-chunk engine kernels, fp32 population storage.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_resident_fp32(int set_id, int N, const ResidentLaunch& L, cudaStream_t st) {
    return engine_resident_t<float>(set_id, N, L, st);
}

int engine_resident_attr_fp32(int set_id, int N, size_t smem) {
    return engine_resident_attr_t<float>(set_id, N, smem);
}

}  // namespace lbm
