// Batched stepping and serving (placeholder until the persistent kernel lands).
#include "rk_internal.h"
using namespace rk;
extern "C" {
rk_status rk_integrate_batch(rk_problem**, int, double, int, rk_stats*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_server_create(size_t, int, rk_server**) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_submit_job(rk_server*, const rk_problem_desc*, const rk_solver_desc*, int, const double*, const double*,
                        const double*, const double*, double, int, uint64_t*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_poll_job(rk_server*, uint64_t, int*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_wait_job(rk_server*, uint64_t, double*, rk_stats*, double*) { set_error("not built yet"); return RK_ERR_ARG; }
rk_status rk_server_destroy(rk_server*) { set_error("not built yet"); return RK_ERR_ARG; }
}
