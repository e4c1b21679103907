// Instantiations of the parent kernel and the persistent replica kernel for
// float state (bd_window.cuh, bd_window2.cuh, bd_persist.cuh). Compiled with
// -fmad=false.
#include "bd_persist.cuh"
#include "bd_launch.h"
#include "bd_variants.h"

namespace bdra {

namespace {
template <int L> const void* parent_fn(bool lj)
{
    return lj ? (const void*)parent_kernel<float, L, true, true> : (const void*)parent_kernel<float, L, true, false>;
}
}  // namespace

#define BD_PARENT_TILES(X) X(2) X(4) X(7) X(10) X(13) X(16)

const void* parent_func_f32(int L, bool lj)
{
    switch (L) {
#define X(l) case l: return parent_fn<l>(lj);
        BD_PARENT_TILES(X)
#undef X
    default: return nullptr;
    }
}

const void* persist_plain_f32(int v)
{
    switch (v) {
#define X(x) case x: return (const void*)replica_persist_kernel<float, true, x, false>;
        BD_VARIANTS_F32_MAIN(X)
#undef X
    default: return persist_more_f32(v, false);
    }
}

const void* persist_func_f32(int v, bool conf)
{
    return conf ? persist_conf_f32(v) : persist_plain_f32(v);
}

int persist_threads_f32() { return Persist<float>::threads; }

size_t persist_smem_f32(int v)
{
    switch (v) {
#define X(x) case x: return PersistSmem<float, true, x>::bytes;
        BD_VARIANTS_F32(X)
#undef X
    default: return 0;
    }
}

// Occupancy with the variant's dynamic shared memory, which is also allowed
// here (above the default 48 KiB) for the current device.
cudaError_t persist_blocks_per_sm_f32(int v, bool conf, int* n)
{
    const void* f = persist_func_f32(v, conf);
    if (!f) return cudaErrorInvalidValue;
    const size_t smem = persist_smem_f32(v);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, f, Persist<float>::threads, smem);
}

}  // namespace bdra
