// The compiled step variants of the persistent replica kernel (ItemDev::variant;
// kVariantsF32 / kVariantsF64 in bd_launch.h list the same), as X-macros for
// the instantiation units.
#pragma once
#define BD_VARIANTS_F32(X) X(4) X(7) X(10) X(13) X(16) X(kPairBase + 4) X(kPairBase + 7) \
    X(kLJBase + 2) X(kLJBase + 4) X(kLJBase + 5) X(kLJBase + 7) X(kLJBase + 16)
#define BD_VARIANTS_F64(X) X(2) X(4) X(7) X(10) X(13) X(16) \
    X(kLJBase + 2) X(kLJBase + 4) X(kLJBase + 5) X(kLJBase + 7) X(kLJBase + 16)
