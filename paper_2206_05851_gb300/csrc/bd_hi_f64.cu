// Instantiations of the hydrodynamic-interaction kernels (bd_hi.cuh) for
// double state, for chains of up to kHISmallBeads beads and of up to
// kHIMaxBeads. Compiled with -fmad=false.
#include "bd_hi.cuh"
#include "bd_launch.h"

namespace bdra {

static_assert(kHIThreads == kHIThreadsHost && kHIMaxBeads == kHIMaxBeadsHost &&
              kHISmallBeads == kHISmallBeadsHost, "HI launch constants");

const void* hi_replica_func_f64(bool small)
{
    return small ? (const void*)hi_replica_kernel<double, false, kHINTSmall>
                 : (const void*)hi_replica_kernel<double, false, kHINTMax>;
}
const void* hi_parent_func_f64(bool small)
{
    return small ? (const void*)hi_parent_kernel<double, false, kHINTSmall>
                 : (const void*)hi_parent_kernel<double, false, kHINTMax>;
}
size_t hi_smem_f64(bool small)
{
    return small ? sizeof(HIShared<double, kHINTSmall>) : sizeof(HIShared<double, kHINTMax>);
}

int hi_threads_f64(bool)
{
    return kHIThreads;
}

cudaError_t hi_prepare_f64()
{
    for (int small = 0; small < 2; ++small) {
        const int smem = (int)hi_smem_f64(small);
        cudaError_t e = cudaFuncSetAttribute(hi_replica_func_f64(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(hi_parent_func_f64(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bdra
