// Fused dslash + clover kernels, F64 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(F64)
WCL_DEFINE_MRHS_LAUNCHER(F64)
}  // namespace wcl
