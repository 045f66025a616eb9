// Nodal projection (Step 11; Eq. div3; Appendix A) -- placeholder until the
// nodal kernels land.
#include "mx_solver.cuh"

mx_status nodal_apply(mx_ctx *c, const mx_geom *, int, const double *, const double *, const double *, const double *,
                      double *, double *) {
    return set_err(c, MX_ERR_ARG, "nodal operator not built yet");
}
void destroy_nodal_plans(mx_ctx *) {}
void destroy_batch_plan(mx_ctx *) {}

extern "C" mx_status mx_nodal_project(mx_ctx *c, const mx_geom *, double *, double *, double *, const double *,
                                      const double *, const double *, double *, const mx_opts *, mx_info *) {
    return set_err(c, MX_ERR_ARG, "nodal projection not built yet");
}
extern "C" mx_status mx_mac_project_batched(mx_ctx *c, int, const mx_geom *, double *const *, double *const *,
                                            double *const *, const double *const *, const double *const *,
                                            const double *const *, double *const *, const mx_opts *, mx_info *) {
    return set_err(c, MX_ERR_ARG, "batched projection not built yet");
}
