// Packed-pair multi-RHS dslash + clover kernels (two right-hand sides per thread), F16 storage.
#include "dslash_pair.cuh"

namespace wcl {
WCL_DEFINE_PAIR_LAUNCHER(F16)
}  // namespace wcl
