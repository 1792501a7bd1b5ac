// Fused dslash + clover in double-float arithmetic on the FP64 fields.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS_DF(DF64)
}  // namespace wcl
