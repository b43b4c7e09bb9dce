// Engine kernels with fp32 population storage.
#include "engine_launch.cuh"

namespace lbm {

__global__ void k_engine_advance(unsigned int* seed, unsigned int by) { *seed += by; }

cudaError_t engine_step_fp32(int set_id, int N, const EngineLaunch& L, cudaStream_t st) {
    return engine_step_t<float>(set_id, N, L, st);
}

int engine_occupancy_fp32(int set_id, int N) { return engine_occupancy_t<float>(set_id, N); }

cudaError_t engine_reduce(const void* solves, const int* active, double* out, int nslots,
                          cudaStream_t st) {
    k_engine_reduce<float><<<nslots, 256, 0, st>>>(static_cast<const EngineSolve<float>*>(solves),
                                                   active, out);
    return cudaGetLastError();
}

cudaError_t engine_advance(unsigned int* seed, unsigned int by, cudaStream_t st) {
    k_engine_advance<<<1, 1, 0, st>>>(seed, by);
    return cudaGetLastError();
}

}  // namespace lbm
