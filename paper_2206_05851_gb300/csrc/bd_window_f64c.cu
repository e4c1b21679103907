// Instantiations of the persistent replica kernel for double state with the
// Eq. 5 window-end diagnostics compiled in (BD_FLAG_CONFORMATION); kept in
// their own unit so that the plain kernels (bd_window_f64.cu) are untouched
// by them. Compiled with -fmad=false.
#include "bd_persist.cuh"
#include "bd_launch.h"
#include "bd_variants.h"

namespace bdra {

const void* persist_conf_f64(int v)
{
    switch (v) {
#define X(x) case x: return (const void*)replica_persist_kernel<double, false, x, true>;
        BD_VARIANTS_F64(X)
#undef X
    default: return nullptr;
    }
}

}  // namespace bdra
