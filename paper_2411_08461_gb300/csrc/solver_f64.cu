// Krylov driver with F64 inner (sloppy) precision.
#include "solver.cuh"

namespace wcl {
template wcl_status krylov_solve<F64>(const std::vector<wcl_ctx*>&, int, const wcl_solve_params&, const SolveIO&,
                                     wcl_solve_info*);
}  // namespace wcl
