// Fused dslash + clover kernels, F64 storage.
#include "dslash.cuh"

namespace wcl {
WCL_DEFINE_DSLASH_LAUNCHERS(F64)
WCL_DEFINE_MRHS_LAUNCHER(F64)

// Under lazy module loading a module is loaded -- its code placed in device memory --
// on the first use of one of its kernels; asking for a kernel's attributes does that
// without a launch.  Used to load this module before wcl_apply_Mpc_noalloc runs it.
cudaError_t load_dslash_f64_module() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, dslash_kernel<F64, false, MODE_POST, EPI_NONE>);
}
}  // namespace wcl
