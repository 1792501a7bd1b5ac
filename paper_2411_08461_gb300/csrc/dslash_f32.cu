// Fused dslash + clover kernels, F32 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(F32)
WCL_DEFINE_MRHS_LAUNCHER(F32)
}  // namespace wcl
