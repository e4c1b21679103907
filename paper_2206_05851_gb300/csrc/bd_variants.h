// The compiled step variants of the persistent replica kernel (ItemDev::variant;
// kVariantsF32 / kVariantsF64 in bd_launch.h list the same), as X-macros for
// the instantiation units.
#pragma once
// Float32: the main set (instantiated in bd_window_f32.cu / bd_window_f32c.cu)
// and the in-between tiles (bd_window_f32b.cu), which the planner takes for
// bead counts the main tiles fit with more idle lanes or spring slots.
#define BD_VARIANTS_F32_MAIN(X) X(4) X(7) X(10) X(13) X(16) X(kPairBase + 4) X(kPairBase + 7) \
    X(kLJBase + 2) X(kLJBase + 4) X(kLJBase + 5) X(kLJBase + 7) X(kLJBase + 16)
#define BD_VARIANTS_F32_MORE(X) X(5) X(6) X(8) X(9) X(11) X(12) X(14) X(15) \
    X(kPairBase + 5) X(kPairBase + 6)
#define BD_VARIANTS_F32(X) BD_VARIANTS_F32_MAIN(X) BD_VARIANTS_F32_MORE(X)
#define BD_VARIANTS_F64(X) X(2) X(4) X(7) X(10) X(13) X(16) \
    X(kLJBase + 2) X(kLJBase + 4) X(kLJBase + 5) X(kLJBase + 7) X(kLJBase + 16)
