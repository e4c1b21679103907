// Instantiations of the parent and replica kernels for float state
// (see bd_window.cuh). Compiled with -fmad=false.
#include "bd_window.cuh"
#include "bd_window2.cuh"
#include "bd_launch.h"

namespace bdra {

namespace {
template <int L>
cudaError_t launch_rep(int grid, int threads, size_t smem, cudaStream_t st, const StepParams& p)
{
    replica_kernel<float, L, true><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}
template <int L>
cudaError_t launch_par(int grid, int threads, cudaStream_t st, const StepParams& p)
{
    parent_kernel<float, L, true><<<grid, threads, 0, st>>>(p);
    return cudaGetLastError();
}
template <int L>
cudaError_t launch_rep2(int grid, int threads, size_t smem, cudaStream_t st, const StepParams& p)
{
    replica2_kernel<L><<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}
template <int L>
cudaError_t prepare_rep2(size_t smem)
{
    return cudaFuncSetAttribute(replica2_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}
template <int L>
cudaError_t prepare_rep(size_t smem, cudaFuncAttributes* attr)
{
    cudaError_t e = cudaFuncSetAttribute(replica_kernel<float, L, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return attr ? cudaFuncGetAttributes(attr, replica_kernel<float, L, true>) : cudaSuccess;
}
}  // namespace

#define BD_TILES(X) X(2) X(4) X(7) X(10) X(13) X(16)

cudaError_t launch_replica_f32(int L, int grid, int threads, size_t smem, cudaStream_t st,
                                const StepParams& p)
{
    switch (L) {
#define X(l) case l: return launch_rep<l>(grid, threads, smem, st, p);
        BD_TILES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_parent_f32(int L, int grid, int threads, cudaStream_t st, const StepParams& p)
{
    switch (L) {
#define X(l) case l: return launch_par<l>(grid, threads, st, p);
        BD_TILES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_replica_f32(int L, size_t smem, cudaFuncAttributes* attr)
{
    switch (L) {
#define X(l) case l: return prepare_rep<l>(smem, attr);
        BD_TILES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

#define BD_PAIR_TILES(X) X(4) X(7)

cudaError_t launch_replica2_f32(int L, int grid, int threads, size_t smem, cudaStream_t st,
                                const StepParams& p)
{
    switch (L) {
#define X(l) case l: return launch_rep2<l>(grid, threads, smem, st, p);
        BD_PAIR_TILES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_replica2_f32(int L, size_t smem)
{
    switch (L) {
#define X(l) case l: return prepare_rep2<l>(smem);
        BD_PAIR_TILES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

int max_threads_f32() { return Tile<float, 2>::max_threads; }

}  // namespace bdra
