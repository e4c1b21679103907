// Instantiations of the hydrodynamic-interaction kernels (bd_hi.cuh) for
// double state. Compiled with -fmad=false.
#include "bd_hi.cuh"
#include "bd_launch.h"

namespace bdra {

static_assert(kHIThreads == kHIThreadsHost && kHIMaxBeads == kHIMaxBeadsHost, "HI launch constants");

const void* hi_replica_func_f64() { return (const void*)hi_replica_kernel<double, false>; }
const void* hi_parent_func_f64() { return (const void*)hi_parent_kernel<double, false>; }
size_t hi_smem_f64() { return sizeof(HIShared<double>); }

cudaError_t hi_prepare_f64()
{
    const int smem = (int)sizeof(HIShared<double>);
    cudaError_t e = cudaFuncSetAttribute(hi_replica_kernel<double, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(hi_parent_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace bdra
