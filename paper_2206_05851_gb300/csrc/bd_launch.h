// Host-visible entry points of the per-precision kernel units.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include "bd_device.cuh"

namespace bdra {

static const int kTiles[] = {2, 4, 7, 10, 13, 16};   // springs per lane
static const int kNumTiles = 6;
// springs per lane with two replicas per lane (larger tiles spill at 128 registers)
static const int kPairTiles[] = {4, 7};
static const int kNumPairTiles = 2;

cudaError_t launch_replica_f32(int L, int grid, int threads, size_t smem, cudaStream_t st,
                               const StepParams& p);
cudaError_t launch_replica_f64(int L, int grid, int threads, size_t smem, cudaStream_t st,
                               const StepParams& p);
cudaError_t launch_parent_f32(int L, int grid, int threads, cudaStream_t st, const StepParams& p);
cudaError_t launch_parent_f64(int L, int grid, int threads, cudaStream_t st, const StepParams& p);
cudaError_t prepare_replica_f32(int L, size_t smem, cudaFuncAttributes* attr);
cudaError_t prepare_replica_f64(int L, size_t smem, cudaFuncAttributes* attr);
cudaError_t launch_replica2_f32(int L, int grid, int threads, size_t smem, cudaStream_t st,
                                const StepParams& p);
cudaError_t prepare_replica2_f32(int L, size_t smem);
int max_threads_f32();
int max_threads_f64();

}  // namespace bdra
