// Instantiations of the hydrodynamic-interaction kernels (bd_hi.cuh) for
// float state, for chains of up to kHISmallBeads beads and of up to
// kHIMaxBeads. Compiled with -fmad=false.
#include "bd_hi.cuh"
#include "bd_launch.h"

namespace bdra {

static_assert(kHIThreads == kHIThreadsHost && kHIMaxBeads == kHIMaxBeadsHost &&
              kHISmallBeads == kHISmallBeadsHost, "HI launch constants");

const void* hi_replica_func_f32(bool small)
{
    return small ? (const void*)hi_replica_kernel<float, true, kHINTSmall>
                 : (const void*)hi_replica_kernel<float, true, kHINTMax>;
}
const void* hi_parent_func_f32(bool small)
{
    return small ? (const void*)hi_parent_kernel<float, true, kHINTSmall>
                 : (const void*)hi_parent_kernel<float, true, kHINTMax>;
}
size_t hi_smem_f32(bool small)
{
    return small ? sizeof(HIShared<float, kHINTSmall>) : sizeof(HIShared<float, kHINTMax>);
}

cudaError_t hi_prepare_f32()
{
    for (int small = 0; small < 2; ++small) {
        const int smem = (int)hi_smem_f32(small);
        cudaError_t e = cudaFuncSetAttribute(hi_replica_func_f32(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(hi_parent_func_f32(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bdra
