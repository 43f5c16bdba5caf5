// stage.cu -- the staging kernel: one CTA of 1024 threads per problem (grid =
// number of problems), its scratch in shared memory; the staging itself is
// stage_run in stage_dev.cuh.
#include <cstdint>

#include "stage_dev.cuh"

namespace rei {

constexpr uint32_t kStageBytesSmem = 32 * 1024;  // strings up to this total are staged from shared memory

__global__ void __launch_bounds__(kStageThreads, 1) k_stage(const StageJob *jobs) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    StageSmem M;
    stage_layout(kMaxIC, kStageBytesSmem, smem_raw, &M);
    stage_run(jobs[blockIdx.x], M);
}

size_t stage_smem_bytes() { return stage_layout(kMaxIC, kStageBytesSmem, nullptr, nullptr); }

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
