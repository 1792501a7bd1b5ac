// Packed-pair multi-RHS dslash + clover kernels (two right-hand sides per thread), F32 storage.
#include "dslash_pair.cuh"

namespace wcl {
WCL_DEFINE_PAIR_LAUNCHER(F32)
}  // namespace wcl
