// Host-visible entry points of the per-precision kernel units.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include "bd_device.cuh"

namespace bdra {

// Parent-kernel tiles (springs per lane).
static const int kTiles[] = {2, 4, 7, 10, 13, 16};
static const int kNumTiles = 6;

// Replica step variants compiled into the persistent kernel (ItemDev::variant):
// float32: one replica per lane with 4..16 springs, two replicas per lane
// with 4..7 springs (larger pair tiles spill at 128 registers);
// float64: one replica per lane with 2..16 springs; both precisions: the
// collapsed-chain step (harmonic springs, Lennard-Jones pair forces) with 2,
// 4, 5, 7 or 16 springs per lane (5: the paper's 50-bead chain fills ten
// lanes exactly). (bd_variants.h lists the same.)
static const int kVariantsF32[] = {4, 7, 10, 13, 16, kPairBase + 4, kPairBase + 7,
                                   kLJBase + 2, kLJBase + 4, kLJBase + 5, kLJBase + 7, kLJBase + 16,
                                   5, 6, 8, 9, 11, 12, 14, 15, kPairBase + 5, kPairBase + 6};
static const int kNumVariantsF32 = 22;
static const int kVariantsF64[] = {2, 4, 7, 10, 13, 16,
                                   kLJBase + 2, kLJBase + 4, kLJBase + 5, kLJBase + 7, kLJBase + 16};
static const int kNumVariantsF64 = 11;

// Variant codes are below kVariantCodes (cost tables are indexed by code).
// kHIBase (hydrodynamic interaction, one CTA per replica) is not a tile
// variant: the planner gives it to every chain with an RPY radius.
constexpr int kVariantCodes = kHIBase + 2;

// kHIBase: chains of up to kHISmallBeadsHost beads (fewer tiles per thread,
// three CTAs per SM in float32); kHIBase + 1: up to kHIMaxBeadsHost.
inline bool variant_hi(int v) { return v >= kHIBase; }
inline bool variant_lj(int v) { return v >= kLJBase && v < kHIBase; }
inline bool variant_paired(int v) { return v >= kPairBase && v < kLJBase; }
inline int variant_tile(int v)
{
    return v >= kHIBase ? 0 : v >= kLJBase ? v - kLJBase : v >= kPairBase ? v - kPairBase : v;
}

// Hydrodynamic interaction (bd_hi.cuh; bd_hi_f32.cu, bd_hi_f64.cu): kernels,
// their CTA size and bead limit, the dynamic shared memory of a CTA, and the
// one-time attribute set-up that allows it.
constexpr int kHIThreadsHost = 256;
constexpr int kHIMaxBeadsHost = 64;
constexpr int kHISmallBeadsHost = 50;
const void* hi_replica_func_f32(bool small);
const void* hi_replica_func_f64(bool small);
const void* hi_parent_func_f32(bool small);
const void* hi_parent_func_f64(bool small);
size_t hi_smem_f32(bool small);
size_t hi_smem_f64(bool small);
int hi_threads_f32(bool small);        // threads of a CTA of these kernels
int hi_threads_f64(bool small);
cudaError_t hi_prepare_f32();
cudaError_t hi_prepare_f64();

// Parent kernels per tile; lj: the collapsed-chain step.
const void* parent_func_f32(int L, bool lj);
const void* parent_func_f64(int L, bool lj);
const void* persist_plain_f32(int variant);     // without the Eq. 5 diagnostics
const void* persist_plain_f64(int variant);
const void* persist_conf_f32(int variant);      // with them (bd_window_f32c.cu)
const void* persist_more_f32(int variant, bool conf);   // the in-between tiles (bd_window_f32b.cu)
const void* persist_conf_f64(int variant);
const void* persist_func_f32(int variant, bool conf);
const void* persist_func_f64(int variant, bool conf);
int persist_threads_f32();
int persist_threads_f64();
cudaError_t persist_blocks_per_sm_f32(int variant, bool conf, int* n);
cudaError_t persist_blocks_per_sm_f64(int variant, bool conf, int* n);
size_t persist_smem_f32(int variant);     // dynamic shared memory per CTA
size_t persist_smem_f64(int variant);

// Adjoint kernels (bd_adjoint.cuh), launched with kAdjThreads threads (bd_device.cuh): the
// parent kernels exist for every tile of kTiles, the replica-window kernel
// for the tiles of kAdjTiles.
enum { ADJ_PARENT_RECOMPUTE = 0, ADJ_REPLICA_WINDOW = 1, ADJ_PARENT_BACKWARD = 2 };
static const int kAdjTiles[] = {4, 7, 16};
static const int kNumAdjTiles = 3;
const void* adj_func_f32(int kind, int L);
const void* adj_func_f64(int kind, int L);

}  // namespace bdra
