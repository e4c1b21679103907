// The persistent replica kernels: every warp claims work items (chain,
// replica group) from its launch's queue, longest first, until none is left.
// Warps are independent - a warp's replicas, their window-end reduction and
// their state never involve another warp - so chains of any bead and replica
// count share a launch and the load balances at warp granularity. There is
// one kernel per step variant (springs per lane, one or two replicas per
// lane), so that each gets its own register allocation; a step launches one
// per variant present, as parallel branches of one CUDA graph.
#pragma once

#include "bd_window.cuh"
#include "bd_window2.cuh"

namespace bdra {

template <typename T> struct Persist {
    static constexpr int threads = (sizeof(T) == 4) ? BD_F32_THREADS : BD_F64_THREADS;
};

// Dynamic shared memory of one CTA: per warp the window-end scratch
// (kWarpScratch values) and, for the float32 variants, the table of
// per-bead Philox parts (32 L entries: every bead a lane of a chain that fits
// the tile draws).
template <typename T, bool FAST, int V> struct PersistSmem {
    static constexpr int L = V >= kLJBase ? V - kLJBase : (V >= kPairBase ? V - kPairBase : V);
    static constexpr bool tab = sizeof(T) == 4 && FAST;
    static constexpr int warps = Persist<T>::threads / 32;
    static constexpr size_t wsm_bytes = (size_t)warps * kWarpScratch * sizeof(T);
    static constexpr int tab_per_warp = tab ? 32 * L : 0;
    static constexpr size_t bytes = wsm_bytes + (size_t)warps * tab_per_warp * sizeof(uint4);
    static_assert(wsm_bytes % 16 == 0, "table must start 16-byte aligned");
    // window-end scratch: replicas per warp x springs <= (2 if paired) x 32 L
    static_assert(((V >= kPairBase && V < kLJBase) ? 64 : 32) * L <= kWarpScratch,
                  "window scratch too small for the tile");
};

template <typename T, bool FAST, int V, bool CONF = false>
__global__ void __launch_bounds__(Persist<T>::threads, 1) replica_persist_kernel(const StepParams p)
{
    using SM = PersistSmem<T, FAST, V>;
    extern __shared__ uint4 bd_smem[];
    const int warp = threadIdx.x >> 5;
    T* wsm = reinterpret_cast<T*>(bd_smem) + warp * kWarpScratch;
    uint4* ptab = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(bd_smem) + SM::wsm_bytes) +
                  warp * SM::tab_per_warp;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(p.queue, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= p.n_items) break;
        if constexpr (V >= kLJBase)
            run_one_item<T, V - kLJBase, FAST, SM::tab, CONF, true>(p.items[idx], p, wsm, ptab);
        else if constexpr (V >= kPairBase)
            run_pair_item<V - kPairBase, SM::tab, CONF>(p.items[idx], p, wsm, ptab);
        else
            run_one_item<T, V, FAST, SM::tab, CONF>(p.items[idx], p, wsm, ptab);
    }
}

}  // namespace bdra
