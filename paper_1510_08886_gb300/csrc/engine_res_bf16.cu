// Resident-chunk engine kernels, bfloat16 population storage.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_resident_bf16(int set_id, int N, const ResidentLaunch& L, cudaStream_t st) {
    return engine_resident_t<__nv_bfloat16>(set_id, N, L, st);
}

int engine_resident_attr_bf16(int set_id, int N, size_t smem) {
    return engine_resident_attr_t<__nv_bfloat16>(set_id, N, smem);
}

}  // namespace lbm
