// Fused dslash + clover kernels, BF16 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(BF16)
WCL_DEFINE_MRHS_LAUNCHER(BF16)
}  // namespace wcl
