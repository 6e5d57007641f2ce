// Explicit stages of the step (Sec. III A-B): viscosity, cell pressure
// gradient, stress divergence, Godunov edge states, MAC divergence/correction,
// convective term and viscous right-hand side, nodal divergence and the
// projection update.  One thread per cell (or face, or node), grid-stride.
//
// This unit is compiled without FMA contraction: the predictor takes upwind
// decisions on the sign of computed values, and keeping every product rounded
// separately keeps those decisions aligned with a plain FP64 evaluation.
#include "hb_explicit.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define HB_DISPATCH(dim, KERNEL, GRID, ...)                            \
  do {                                                                \
    if ((dim) == 2)                                                   \
      launch(c, kSlotExplicit, KERNEL<2>, (GRID), kThreads, __VA_ARGS__); \
    else                                                              \
      launch(c, kSlotExplicit, KERNEL<3>, (GRID), kThreads, __VA_ARGS__); \
  } while (0)

int launch_eta(hbf_ctx* c) {
  HB_DISPATCH(c->dim, k_eta, grid_for(c->g.ncell), c->u, c->eta, c->g, c->rheo);
  return cuda_check(c, cudaGetLastError(), "k_eta");
}

int launch_eta_faces(hbf_ctx* c) {
  for (int a = 0; a < c->dim; ++a)
    HB_DISPATCH(c->dim, k_eta_faces, grid_for(c->g.nface[a]), c->eta, c->lv[0].ef[a], a, c->g);
  return cuda_check(c, cudaGetLastError(), "k_eta_faces");
}

int launch_predict(hbf_ctx* c, double dt) {
  const Geom& g = c->g;
  Force fo{{c->f[0], c->f[1], c->f[2]}};
  HB_DISPATCH(c->dim, k_grad_p, grid_for(g.ncell), c->p, c->Gp, g);
  int st = launch_eta_faces(c);
  if (st) return st;
  if ((st = tensor_lu(c, c->u, c->Lu))) return st;
  HB_DISPATCH(c->dim, k_slopes, grid_for(g.ncell), c->u, c->slopes, g);
  const StepC k = step_consts(g, c->dim, dt, c->rho, c->theta);
  HB_DISPATCH(c->dim, k_hats, grid_for(g.ncell), c->u, c->slopes, c->Gp, c->Lu, fo, c->predictor_visc, c->hats,
              c->tcom, g, k);
  for (int a = 0; a < c->dim; ++a)
    HB_DISPATCH(c->dim, k_traces, grid_for(g.nface[a]), c->u, c->slopes, c->tcom, a, c->uL[a], c->uR[a],
                c->uadv[a], g, k);
  return cuda_check(c, cudaGetLastError(), "predict kernels");
}

int launch_mac_rhs(hbf_ctx* c, double* rhs) {
  HB_DISPATCH(c->dim, k_mac_rhs, grid_for(c->g.ncell), c->uadv[0], c->uadv[1], c->uadv[2], rhs, c->g);
  return cuda_check(c, cudaGetLastError(), "k_mac_rhs");
}

int launch_mac_correct(hbf_ctx* c, const double* phi) {
  for (int a = 0; a < c->dim; ++a)
    HB_DISPATCH(c->dim, k_mac_correct, grid_for(c->g.nface[a]), c->uadv[a], phi, c->umac[a], a, c->g);
  return cuda_check(c, cudaGetLastError(), "k_mac_correct");
}

int launch_advect_rhs(hbf_ctx* c, double dt) {
  Force fo{{c->f[0], c->f[1], c->f[2]}};
  HB_DISPATCH(c->dim, k_advect_rhs, grid_for(c->g.ncell), c->u, c->uL[0], c->uL[1], c->uL[2], c->uR[0],
              c->uR[1], c->uR[2], c->umac[0], c->umac[1], c->umac[2], c->Gp, c->Lu, fo, c->rhs, c->g,
              step_consts(c->g, c->dim, dt, c->rho, c->theta));
  return cuda_check(c, cudaGetLastError(), "k_advect_rhs");
}

int launch_nodal_rhs(hbf_ctx* c, double dt, const double* ustar, const double* p, double* out) {
  const StepC k = step_consts(c->g, c->dim, dt, c->rho, c->theta);
  HB_DISPATCH(c->dim, k_grad_p_w, grid_for(c->g.ncell), p, ustar, c->Gp, c->wn, c->g, k);
  HB_DISPATCH(c->dim, k_nodal_rhs, grid_for(c->g.nnode), (const double*)c->wn, out, c->g, k);
  return cuda_check(c, cudaGetLastError(), "k_nodal_rhs");
}

int launch_project_update(hbf_ctx* c, double dt, double* u, const double* p_old, const double* phi) {
  (void)p_old;  // G p^{m-1/2} is still in c->Gp from launch_nodal_rhs
  HB_DISPATCH(c->dim, k_project_update, grid_for(c->g.ncell), u, c->Gp, phi, c->g,
              step_consts(c->g, c->dim, dt, c->rho, c->theta));
  return cuda_check(c, cudaGetLastError(), "k_project_update");
}

}  // namespace hb
