// Fused dslash + clover kernels, F64 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(F64)
}  // namespace wcl
