// Block-AMEn KKT solve (steps a6..a8): placeholder until the solver lands.
#include "iga_internal.cuh"

using namespace iga;

extern "C" void iga_solve_opts_default(iga_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->inner_tol = 1e-3;
  o->max_sweeps = 8;
  o->kick_rank = 4;
  o->rmax = 128;
  o->local_maxit = 200;
  o->refine_max = 6;
  o->precision = IGA_FP32;
  o->verbose = 0;
}

extern "C" iga_status iga_kkt_solve_amen(iga_ctx* ctx, const iga_op*, const iga_op*, const iga_tt*,
                                         double, const iga_solve_opts*, double*, double*, double*,
                                         iga_solve_info*) {
  if (!ctx) return IGA_EINVAL;
  set_error(ctx, "iga_kkt_solve_amen: solver not built in this revision");
  return IGA_EINVAL;
}
