// Instantiations of the persistent replica kernel for float state with the
// Eq. 5 window-end diagnostics compiled in (BD_FLAG_CONFORMATION); kept in
// their own unit so that the plain kernels (bd_window_f32.cu) are untouched
// by them. Compiled with -fmad=false.
#include "bd_persist.cuh"
#include "bd_launch.h"
#include "bd_variants.h"

namespace bdra {

const void* persist_conf_f32(int v)
{
    switch (v) {
#define X(x) case x: return (const void*)replica_persist_kernel<float, true, x, true>;
        BD_VARIANTS_F32_MAIN(X)
#undef X
    default: return persist_more_f32(v, true);
    }
}

}  // namespace bdra
