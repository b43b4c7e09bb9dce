// Cluster-split resident engine kernels, bfloat16 population storage.
#include "engine_launch.cuh"

namespace lbm {

cudaError_t engine_cluster_bf16(int set_id, int N, const ClusterLaunch& L, cudaStream_t st) {
    return engine_cluster_t<__nv_bfloat16>(set_id, N, L, st);
}

int engine_cluster_attr_bf16(int set_id, int N, size_t smem) {
    return engine_cluster_attr_t<__nv_bfloat16>(set_id, N, smem);
}

}  // namespace lbm
