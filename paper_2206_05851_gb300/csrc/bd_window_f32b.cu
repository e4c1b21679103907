// Instantiations of the persistent replica kernel for float state with the
// in-between tiles (BD_VARIANTS_F32_MORE: one replica per lane with 5, 6, 8,
// 9, 11, 12, 14 or 15 springs, two replicas per lane with 5 or 6), with and
// without the Eq. 5 diagnostics; a unit of their own so that they compile in
// parallel with the main set. Compiled with -fmad=false.
#include "bd_persist.cuh"
#include "bd_launch.h"
#include "bd_variants.h"

namespace bdra {

const void* persist_more_f32(int v, bool conf)
{
    switch (v) {
#define X(x) case x: return conf ? (const void*)replica_persist_kernel<float, true, x, true> \
                                 : (const void*)replica_persist_kernel<float, true, x, false>;
        BD_VARIANTS_F32_MORE(X)
#undef X
    default: return nullptr;
    }
}

}  // namespace bdra
