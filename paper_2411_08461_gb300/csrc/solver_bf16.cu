// Krylov driver with BF16 inner (sloppy) precision.
#include "solver.cuh"

namespace wcl {
template wcl_status krylov_solve<BF16>(const std::vector<wcl_ctx*>&, int, const wcl_solve_params&, const SolveIO&,
                                     wcl_solve_info*);
}  // namespace wcl
