// Instantiations of the hydrodynamic-interaction kernels (bd_hi.cuh) for
// float state. Compiled with -fmad=false.
#include "bd_hi.cuh"
#include "bd_launch.h"

namespace bdra {

static_assert(kHIThreads == kHIThreadsHost && kHIMaxBeads == kHIMaxBeadsHost, "HI launch constants");

const void* hi_replica_func_f32() { return (const void*)hi_replica_kernel<float, true>; }
const void* hi_parent_func_f32() { return (const void*)hi_parent_kernel<float, true>; }
size_t hi_smem_f32() { return sizeof(HIShared<float>); }

cudaError_t hi_prepare_f32()
{
    const int smem = (int)sizeof(HIShared<float>);
    cudaError_t e = cudaFuncSetAttribute(hi_replica_kernel<float, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(hi_parent_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace bdra
