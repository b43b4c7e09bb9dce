// Launchers of the engine kernels for one storage type (instantiated in
// engine_fp32.cu, engine_fp16.cu, engine_bf16.cu, engine_fp64.cu and the
// engine_res_*.cu files).
#pragma once

#include "engine_kernels.cuh"

namespace lbm {

// Compute type of a storage type: fp64 storage computes in fp64, every
// other format in fp32.
template <typename S> struct ComputeOf { using type = float; };
template <> struct ComputeOf<double> { using type = double; };
template <typename S> using CompOf = typename ComputeOf<S>::type;

struct EngineLaunch {
    const void* solves;        // EngineSolve<C>* (C the compute type)
    const EngineTile* tiles;   // all tiles
    const int* ntiles;         // device count of this group's tiles
    const int* tile_off;       // device offset of this group's tiles
    int* counter;              // work counter of this (step, group)
    const unsigned* seed;
    int parity, emit, chunk;
    int lm;                    // log2 of the sub-tiles per tile
    int grid;
};

template <class SET, int N, typename S>
cudaError_t engine_step_one(const EngineLaunch& L, cudaStream_t st) {
    using C = CompOf<S>;
    k_engine_step<SET, N, S, C><<<L.grid, kBlock, 0, st>>>(
        static_cast<const EngineSolve<C>*>(L.solves), L.tiles, L.ntiles, L.tile_off, L.counter, L.seed,
        L.parity, L.emit, L.chunk, L.lm);
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

struct ResidentLaunch {
    const void* solves;        // EngineSolve<C>*
    const ResBundle* bundles;  // all bundles (each group's largest first)
    const ResChannel* chans;
    const int* nbundles;       // device count of this group's bundles
    const int* bundle_off;     // device offset of this group's bundles
    int* counter;              // bundle counter of this chunk and group
    const unsigned* seed;
    int K;
    int grid;
    size_t smem;               // dynamic shared memory per block
};

template <class SET, int N, typename S>
const void* resident_fn() {
    return reinterpret_cast<const void*>(&k_engine_resident<SET, N, S, CompOf<S>>);
}

template <class SET, int N, typename S>
cudaError_t resident_one(const ResidentLaunch& L, cudaStream_t st) {
    using C = CompOf<S>;
    k_engine_resident<SET, N, S, C><<<L.grid, res_threads<SET, C>(), L.smem, st>>>(
        static_cast<const EngineSolve<C>*>(L.solves), L.bundles, L.chans, L.nbundles, L.bundle_off, L.counter,
        L.seed, L.K);
    return cudaGetLastError();
}

// Opt the resident kernel of (set, N) into `smem` bytes of dynamic shared
// memory and return its resident blocks per SM at that size (0: unusable).
template <class SET, int N, typename S>
int resident_attr_one(size_t smem) {
    const void* fn = resident_fn<SET, N, S>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_engine_resident<SET, N, S, CompOf<S>>,
                                                      res_threads<SET, CompOf<S>>(), smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return b;
}

#define LBM_RES_DISPATCH(CALL)                                              \
    switch (set_id * 3 + (N - 2)) {                                         \
        case 0: return CALL(SetD2V16, 2);                                   \
        case 1: return CALL(SetD2V16, 3);                                   \
        case 2: return CALL(SetD2V16, 4);                                   \
        case 3: return CALL(SetD2V32, 2);                                   \
        case 4: return CALL(SetD2V32, 3);                                   \
        case 5: return CALL(SetD2V32, 4);                                   \
        case 6: return CALL(SetD2V33, 2);                                   \
        case 7: return CALL(SetD2V33, 3);                                   \
        case 8: return CALL(SetD2V33, 4);                                   \
        case 9: return CALL(SetD2V53, 2);                                   \
        case 10: return CALL(SetD2V53, 3);                                  \
        case 11: return CALL(SetD2V53, 4);                                  \
        case 12: return CALL(SetD2V40, 2);                                  \
        case 13: return CALL(SetD2V40, 3);                                  \
        case 14: return CALL(SetD2V40, 4);                                  \
        case 15: return CALL(SetD2V48, 2);                                  \
        case 16: return CALL(SetD2V48, 3);                                  \
        case 17: return CALL(SetD2V48, 4);                                  \
        default: break;                                                     \
    }

template <typename S>
cudaError_t engine_resident_t(int set_id, int N, const ResidentLaunch& L, cudaStream_t st) {
#define LBM_RES_LAUNCH(SET, NN) resident_one<SET, NN, S>(L, st)
    LBM_RES_DISPATCH(LBM_RES_LAUNCH)
#undef LBM_RES_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename S>
int engine_resident_attr_t(int set_id, int N, size_t smem) {
#define LBM_RES_ATTR(SET, NN) resident_attr_one<SET, NN, S>(smem)
    LBM_RES_DISPATCH(LBM_RES_ATTR)
#undef LBM_RES_ATTR
    return 0;
}

// resident blocks per SM of the engine kernel of (set, N)
template <class SET, int N, typename S>
int engine_occ_one() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_engine_step<SET, N, S, CompOf<S>>, kBlock, 0);
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
