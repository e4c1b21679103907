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
    return small ? (const void*)hi_replica_kernel<float, true, kHISmallT>
                 : (const void*)hi_replica_kernel<float, true, kHIMaxT>;
}
const void* hi_parent_func_f32(bool small)
{
    return small ? (const void*)hi_parent_kernel<float, true, kHISmallT>
                 : (const void*)hi_parent_kernel<float, true, kHIMaxT>;
}
size_t hi_smem_f32() { return sizeof(HIShared<float>); }

cudaError_t hi_prepare_f32()
{
    const int smem = (int)sizeof(HIShared<float>);
    for (int small = 0; small < 2; ++small) {
        cudaError_t e = cudaFuncSetAttribute(hi_replica_func_f32(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(hi_parent_func_f32(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bdra
