// Advection-diffusion CSR path (placeholder until the GMRES kernels land).
#include "rk_internal.h"

namespace rk {
struct GmresWork {};
rk_status csr_setup(rk_problem*) { set_error("RK_OP_ADVDIFF_CSR is not built yet"); return RK_ERR_ARG; }
rk_status csr_free(rk_problem*) { return RK_OK; }
rk_status gmres_solve(rk_problem*, double, const double*, RhsScalars*, void*, int, int*, int*) {
  set_error("GMRES is not built yet"); return RK_ERR_ARG;
}
rk_status csr_precond_f64(rk_problem*, double, const double*, double*) { set_error("not built"); return RK_ERR_ARG; }
rk_status csr_apply_f64(rk_problem*, const double*, double*, RhsScalars*) { set_error("not built"); return RK_ERR_ARG; }
rk_status csr_correct_f64(rk_problem*, double, const double*, const void*, double*, RhsScalars*) {
  set_error("not built"); return RK_ERR_ARG;
}
}  // namespace rk
