// Engine kernels with fp64 population storage and fp64 arithmetic: the
// per-step tiled kernel, its occupancy, and the per-slot reductions of fp64
// slot records.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_step_fp64(int set_id, int N, const EngineLaunch& L, cudaStream_t st) {
    return engine_step_t<double>(set_id, N, L, st);
}

int engine_occupancy_fp64(int set_id, int N) { return engine_occupancy_t<double>(set_id, N); }

cudaError_t engine_reduce_fp64(const void* solves, const int* active, double* out, int nslots,
                               cudaStream_t st) {
    k_engine_reduce<double><<<nslots, 256, 0, st>>>(static_cast<const EngineSolve<double>*>(solves),
                                                    active, out);
    return cudaGetLastError();
}

}  // namespace lbm
