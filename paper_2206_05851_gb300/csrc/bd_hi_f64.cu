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
    return small ? (const void*)hi_replica_kernel<double, false, kHISmallT>
                 : (const void*)hi_replica_kernel<double, false, kHIMaxT>;
}
const void* hi_parent_func_f64(bool small)
{
    return small ? (const void*)hi_parent_kernel<double, false, kHISmallT>
                 : (const void*)hi_parent_kernel<double, false, kHIMaxT>;
}
size_t hi_smem_f64() { return sizeof(HIShared<double>); }

cudaError_t hi_prepare_f64()
{
    const int smem = (int)sizeof(HIShared<double>);
    for (int small = 0; small < 2; ++small) {
        cudaError_t e = cudaFuncSetAttribute(hi_replica_func_f64(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(hi_parent_func_f64(small), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bdra
