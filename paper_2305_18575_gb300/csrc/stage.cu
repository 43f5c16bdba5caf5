// stage.cu -- the staging kernel: one CTA of 1024 threads per problem (grid =
// number of problems), its hash set in shared memory; the staging itself is
// stage_run in stage_dev.cuh.
#include <cstdint>

#include "stage_dev.cuh"

namespace rei {

__global__ void __launch_bounds__(kStageThreads, 1) k_stage(const StageJob *jobs) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *hset = reinterpret_cast<uint64_t *>(smem_raw);
    uint16_t *rank_of = reinterpret_cast<uint16_t *>(hset + kHsetCap);
    uint16_t *uniq = rank_of + kHsetCap;
    int16_t *rank_tab = reinterpret_cast<int16_t *>(uniq + kMaxIC);
    stage_run(jobs[blockIdx.x], hset, rank_of, uniq, rank_tab);
}

size_t stage_smem_bytes() {
    return kHsetCap * sizeof(uint64_t) + kHsetCap * sizeof(uint16_t) + kMaxIC * sizeof(uint16_t) +
           256 * sizeof(int16_t);
}

cudaError_t launch_stage(const StageJob *jobs_dev, uint32_t n_jobs, cudaStream_t stream) {
    static bool attr_set = false;
    const size_t smem = stage_smem_bytes();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_stage<<<n_jobs, kStageThreads, smem, stream>>>(jobs_dev);
    return cudaGetLastError();
}

}  // namespace rei
