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

template <typename T, bool FAST, int V>
__global__ void __launch_bounds__(Persist<T>::threads, 1) replica_persist_kernel(const StepParams p)
{
    __shared__ T wsm_all[Persist<T>::threads / 32][kWarpScratch];
    T* wsm = wsm_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(p.queue, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= p.n_items) break;
        if constexpr (V >= kPairBase)
            run_pair_item<V - kPairBase>(p.items[idx], p, wsm);
        else
            run_one_item<T, V, FAST>(p.items[idx], p, wsm);
    }
}

}  // namespace bdra
