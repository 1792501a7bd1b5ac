// Packed-pair multi-RHS dslash + clover kernels (two right-hand sides per thread), BF16 storage.
#include "dslash_pair.cuh"

namespace wcl {
WCL_DEFINE_PAIR_LAUNCHER(BF16)
}  // namespace wcl
