// Instantiations of the hydrodynamic-interaction kernels for float state:
// chains of up to kHISmallBeads beads on the tensor-core kernels
// (bd_hi_tc.cuh; BD_HI_TC=0 builds the CUDA-core tile kernels of bd_hi.cuh
// for them instead), chains of up to kHIMaxBeads on the CUDA-core tile
// kernels. Compiled with -fmad=false.
#include "bd_hi_tc.cuh"
#include "bd_launch.h"

#ifndef BD_HI_TC
#define BD_HI_TC 1
#endif

namespace bdra {

static_assert(kHIThreads == kHIThreadsHost && kHIMaxBeads == kHIMaxBeadsHost &&
              kHISmallBeads == kHISmallBeadsHost && kTCMaxBeads == kHISmallBeadsHost,
              "HI launch constants");

const void* hi_replica_func_f32(bool small)
{
    if (small && BD_HI_TC) return (const void*)hi_tc_replica_kernel;
    return small ? (const void*)hi_replica_kernel<float, true, kHINTSmall>
                 : (const void*)hi_replica_kernel<float, true, kHINTMax>;
}
const void* hi_parent_func_f32(bool small)
{
    if (small && BD_HI_TC) return (const void*)hi_tc_parent_kernel;
    return small ? (const void*)hi_parent_kernel<float, true, kHINTSmall>
                 : (const void*)hi_parent_kernel<float, true, kHINTMax>;
}
size_t hi_smem_f32(bool small)
{
    if (small && BD_HI_TC) return sizeof(HITCShared);
    return small ? sizeof(HIShared<float, kHINTSmall>) : sizeof(HIShared<float, kHINTMax>);
}
int hi_threads_f32(bool small)
{
    return small && BD_HI_TC ? kTCThreads : kHIThreads;
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
