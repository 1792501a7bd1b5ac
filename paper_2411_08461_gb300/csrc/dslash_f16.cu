// Fused dslash + clover kernels, F16 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(F16)
WCL_DEFINE_MRHS_LAUNCHER(F16)
}  // namespace wcl
