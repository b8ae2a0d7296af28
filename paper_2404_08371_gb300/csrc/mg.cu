// Multigrid pieces (Section 8): filled in below as they are built.
#include "hhg_internal.h"

using namespace hhg;

extern "C" int hhg_op_apply_adjoint_coeff(hhg_op_t*, const void*, const void*, void*, int, int, void*) {
  return fail(HHG_E_UNSUPPORTED, "op_apply_adjoint_coeff: not implemented yet");
}
extern "C" int hhg_prolongate(const hhg_mesh_t*, int, int, const void*, void*, int, void*) {
  return fail(HHG_E_UNSUPPORTED, "prolongate: not implemented yet");
}
extern "C" int hhg_restrict(const hhg_mesh_t*, int, int, const void*, void*, int, void*) {
  return fail(HHG_E_UNSUPPORTED, "restrict: not implemented yet");
}
extern "C" int hhg_rhs_sin3_poisson(const hhg_mesh_t*, int, int, double*, void*) {
  return fail(HHG_E_UNSUPPORTED, "rhs: not implemented yet");
}
extern "C" int hhg_l2_error_sin3(const hhg_mesh_t*, int, int, const double*, double*, void*) {
  return fail(HHG_E_UNSUPPORTED, "l2 error: not implemented yet");
}
extern "C" int hhg_cheb_smooth(hhg_op_t*, const void*, void*, const void*, double, double, double, int, int, void*) {
  return fail(HHG_E_UNSUPPORTED, "cheb_smooth: not implemented yet");
}
extern "C" int hhg_power_iteration(hhg_op_t*, const void*, void*, int, int, double*, void*) {
  return fail(HHG_E_UNSUPPORTED, "power_iteration: not implemented yet");
}
extern "C" int hhg_mg_default_opts(hhg_mg_opts_t* o) {
  if (!o) return fail(HHG_E_ARG, "mg_default_opts: null");
  o->nu1 = 2; o->nu2 = 2; o->cheb_order = 2; o->power_iters = 15; o->cheb_lo = 0.1; o->cheb_hi = 1.1;
  o->tol = 1e-10; o->max_iters = 50; o->mixed = 0; o->fmg = 1; o->coarse_level = 0;
  return HHG_OK;
}
extern "C" int hhg_mg_solve(hhg_op_t*, const double*, double*, const hhg_mg_opts_t*, hhg_mg_stats_t*, void*) {
  return fail(HHG_E_UNSUPPORTED, "mg_solve: not implemented yet");
}
