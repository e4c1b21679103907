// Instantiations of the parent kernel and the persistent replica kernel for
// double state (bd_window.cuh, bd_window2.cuh, bd_persist.cuh). Compiled with
// -fmad=false.
#include "bd_persist.cuh"
#include "bd_launch.h"
#include "bd_variants.h"

namespace bdra {

namespace {
template <int L> const void* parent_fn(bool lj)
{
    return lj ? (const void*)parent_kernel<double, L, false, true> : (const void*)parent_kernel<double, L, false, false>;
}
}  // namespace

#define BD_PARENT_TILES(X) X(2) X(4) X(7) X(10) X(13) X(16)

const void* parent_func_f64(int L, bool lj)
{
    switch (L) {
#define X(l) case l: return parent_fn<l>(lj);
        BD_PARENT_TILES(X)
#undef X
    default: return nullptr;
    }
}

const void* persist_plain_f64(int v)
{
    switch (v) {
#define X(x) case x: return (const void*)replica_persist_kernel<double, false, x, false>;
        BD_VARIANTS_F64(X)
#undef X
    default: return nullptr;
    }
}

const void* persist_func_f64(int v, bool conf)
{
    return conf ? persist_conf_f64(v) : persist_plain_f64(v);
}

int persist_threads_f64() { return Persist<double>::threads; }

size_t persist_smem_f64(int v)
{
    switch (v) {
#define X(x) case x: return PersistSmem<double, false, x>::bytes;
        BD_VARIANTS_F64(X)
#undef X
    default: return 0;
    }
}

// Occupancy with the variant's dynamic shared memory, which is also allowed
// here (above the default 48 KiB) for the current device.
cudaError_t persist_blocks_per_sm_f64(int v, bool conf, int* n)
{
    const void* f = persist_func_f64(v, conf);
    if (!f) return cudaErrorInvalidValue;
    const size_t smem = persist_smem_f64(v);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, f, Persist<double>::threads, smem);
}

}  // namespace bdra
