// Instantiations of the adjoint kernels (bd_adjoint.cuh) for double state.
// Compiled with -fmad=false, like the forward kernels, so that the
// recomputed trajectories are bitwise the forward ones.
#include "bd_adjoint.cuh"
#include "bd_launch.h"

namespace bdra {

#define BD_ADJ_PARENT_TILES(X) X(2) X(4) X(7) X(10) X(13) X(16)
#define BD_ADJ_REPLICA_TILES(X) X(4) X(7) X(16)

const void* adj_func_f64(int kind, int L)
{
    switch (kind) {
    case ADJ_PARENT_RECOMPUTE:
        switch (L) {
#define X(l) case l: return (const void*)adj_parent_recompute_kernel<double, l, false>;
            BD_ADJ_PARENT_TILES(X)
#undef X
        }
        break;
    case ADJ_PARENT_BACKWARD:
        switch (L) {
#define X(l) case l: return (const void*)adj_parent_backward_kernel<double, l>;
            BD_ADJ_PARENT_TILES(X)
#undef X
        }
        break;
    case ADJ_REPLICA_WINDOW:
        switch (L) {
#define X(l) case l: return (const void*)adj_replica_window_kernel<double, l, false>;
            BD_ADJ_REPLICA_TILES(X)
#undef X
        }
        break;
    }
    return nullptr;
}

}  // namespace bdra
