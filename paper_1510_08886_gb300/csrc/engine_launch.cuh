// Launchers of the engine kernels for one storage type (instantiated in
// engine_fp32.cu and engine_fp16.cu).
#pragma once

#include "engine_kernels.cuh"

namespace lbm {

struct EngineLaunch {
    const void* solves;        // EngineSolve<float>*
    const EngineTile* tiles;   // this group's tiles
    const int* ntiles;         // device count of this group's tiles
    int* counter;              // work counter of this (step, group)
    const unsigned* seed;
    int parity, emit, chunk;
    int grid;
};

template <class SET, int N, typename S>
cudaError_t engine_step_one(const EngineLaunch& L, cudaStream_t st) {
    k_engine_step<SET, N, S, float><<<L.grid, kBlock, 0, st>>>(
        static_cast<const EngineSolve<float>*>(L.solves), L.tiles, L.ntiles, L.counter, L.seed,
        L.parity, L.emit, L.chunk);
    return cudaGetLastError();
}

template <class SET, typename S>
cudaError_t engine_step_n(int N, const EngineLaunch& L, cudaStream_t st) {
    switch (N) {
        case 2: return engine_step_one<SET, 2, S>(L, st);
        case 3: return engine_step_one<SET, 3, S>(L, st);
        case 4: return engine_step_one<SET, 4, S>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
cudaError_t engine_step_t(int set_id, int N, const EngineLaunch& L, cudaStream_t st) {
    switch (set_id) {
        case 0: return engine_step_n<SetD2V16, S>(N, L, st);
        case 1: return engine_step_n<SetD2V32, S>(N, L, st);
        case 2: return engine_step_n<SetD2V33, S>(N, L, st);
        case 3: return engine_step_n<SetD2V53, S>(N, L, st);
        case 4: return engine_step_n<SetD2V40, S>(N, L, st);
        case 5: return engine_step_n<SetD2V48, S>(N, L, st);
        default: return cudaErrorInvalidValue;
    }
}

// resident blocks per SM of the engine kernel of (set, N)
template <class SET, int N, typename S>
int engine_occ_one() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_engine_step<SET, N, S, float>, kBlock, 0);
    return b;
}

template <typename S>
int engine_occupancy_t(int set_id, int N) {
#define LBM_OCC(ID, SET)                                      \
    if (set_id == ID) {                                       \
        if (N == 2) return engine_occ_one<SET, 2, S>();       \
        if (N == 3) return engine_occ_one<SET, 3, S>();       \
        if (N == 4) return engine_occ_one<SET, 4, S>();       \
    }
    LBM_OCC(0, SetD2V16)
    LBM_OCC(1, SetD2V32)
    LBM_OCC(2, SetD2V33)
    LBM_OCC(3, SetD2V53)
    LBM_OCC(4, SetD2V40)
    LBM_OCC(5, SetD2V48)
#undef LBM_OCC
    return 0;
}

}  // namespace lbm
