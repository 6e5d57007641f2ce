// Batched explicit stages: each stage of Sec. III A-B is one persistent
// launch over the tiles of every cavity (compiled without FMA contraction,
// like the single-cavity unit, so both take identical decisions).
#include "hb_batch_internal.h"
#include "hb_explicit.cuh"

namespace hb {
namespace batch {

template <int D>
struct OpEta {
  struct Arg {
    const double* u;
    double* eta;
    Geom g;
    Rheo r;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_eta_at<D>(a.u, a.eta, a.g, a.r, t); }
};

template <int D>
struct OpEtaFaces {
  struct Arg {
    const double* eta;
    double* ef[3];
    Geom g;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    const int ax = face_axis(a.g, t);
    k_eta_faces_at<D>(a.eta, a.ef[ax], ax, a.g, t);
  }
};

template <int D>
struct OpGradP {
  struct Arg {
    const double* p;
    double* Gp;
    Geom g;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_grad_p_at<D>(a.p, a.Gp, a.g, t); }
};

template <int D>
struct OpSlopes {
  struct Arg {
    const double* u;
    double* slopes;
    Geom g;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_slopes_at<D>(a.u, a.slopes, a.g, t); }
};

template <int D>
struct OpHats {
  struct Arg {
    const double *u, *slopes, *Gp, *Lu;
    Force fo;
    int pv;
    double *hats, *tcom;
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    k_hats_at<D>(a.u, a.slopes, a.Gp, a.Lu, a.fo, a.pv, a.hats, a.tcom, a.g, a.k, t);
  }
};

template <int D>
struct OpTraces {
  struct Arg {
    const double *u, *slopes, *tcom;
    double *uL[3], *uR[3], *uadv[3];
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    const int ax = face_axis(a.g, t);
    k_traces_at<D>(a.u, a.slopes, a.tcom, ax, a.uL[ax], a.uR[ax], a.uadv[ax], a.g, a.k, t);
  }
};

template <int D>
struct OpMacRhs {
  struct Arg {
    const double* ua[3];
    double* rhs;
    Geom g;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_mac_rhs_at<D>(a.ua[0], a.ua[1], a.ua[2], a.rhs, a.g, t); }
};

template <int D>
struct OpMacCorrect {
  struct Arg {
    const double* uadv[3];
    const double* phi;
    double* umac[3];
    Geom g;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    const int ax = face_axis(a.g, t);
    k_mac_correct_at<D>(a.uadv[ax], a.phi, a.umac[ax], ax, a.g, t);
  }
};

template <int D>
struct OpAdvectRhs {
  struct Arg {
    const double* u;
    const double *uL[3], *uR[3], *um[3];
    const double *Gp, *Lu;
    Force fo;
    double* rhs;
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    k_advect_rhs_at<D>(a.u, a.uL[0], a.uL[1], a.uL[2], a.uR[0], a.uR[1], a.uR[2], a.um[0], a.um[1], a.um[2], a.Gp,
                       a.Lu, a.fo, a.rhs, a.g, a.k, t);
  }
};

template <int D>
struct OpGradPW {
  struct Arg {
    const double *p, *ustar;
    double *Gp, *w;
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_grad_p_w_at<D>(a.p, a.ustar, a.Gp, a.w, a.g, a.k, t); }
};

template <int D>
struct OpNodalRhs {
  struct Arg {
    const double* w;
    double* out;
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) { k_nodal_rhs_at<D>(a.w, a.out, a.g, a.k, t); }
};

template <int D>
struct OpProjectUpdate {
  struct Arg {
    double* u;
    const double *Gp, *phi;
    Geom g;
    StepC k;
  };
  static __device__ void apply(const Arg& a, int t, int) {
    k_project_update_at<D>(a.u, a.Gp, a.phi, a.g, a.k, t);
  }
};

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <class Op>
static void* table(hbf_batch* B, const std::vector<typename Op::Arg>& h) {
  return upload_table(B, h);
}

struct ExplicitTables {
  void *eta, *ef, *gp, *gpw, *slopes, *hats, *traces, *macrhs, *maccorr, *advect, *nrhs, *update;
};

template <int D>
static void build_tables(hbf_batch* B, ExplicitTables& T) {
  std::vector<typename OpEta<D>::Arg> a1;
  std::vector<typename OpEtaFaces<D>::Arg> a2;
  std::vector<typename OpGradP<D>::Arg> a3;
  std::vector<typename OpSlopes<D>::Arg> a4;
  std::vector<typename OpHats<D>::Arg> a5;
  std::vector<typename OpTraces<D>::Arg> a6;
  std::vector<typename OpMacRhs<D>::Arg> a7;
  std::vector<typename OpMacCorrect<D>::Arg> a8;
  std::vector<typename OpAdvectRhs<D>::Arg> a9;
  std::vector<typename OpNodalRhs<D>::Arg> a10;
  std::vector<typename OpGradPW<D>::Arg> a12;
  std::vector<typename OpProjectUpdate<D>::Arg> a11;
  for (int i = 0; i < B->ncav; ++i) {
    hbf_ctx* c = B->cav[i];
    const StepC k = step_consts(c->g, D, B->dt[i], c->rho, c->theta);
    Force fo{{c->f[0], c->f[1], c->f[2]}};
    a1.push_back({c->u, c->eta, c->g, c->rheo});
    a2.push_back({c->eta, {c->lv[0].ef[0], c->lv[0].ef[1], c->lv[0].ef[2]}, c->g});
    a3.push_back({c->p, c->Gp, c->g});
    a4.push_back({c->u, c->slopes, c->g});
    a5.push_back({c->u, c->slopes, c->Gp, c->Lu, fo, c->predictor_visc, c->hats, c->tcom, c->g, k});
    a6.push_back({c->u, c->slopes, c->tcom, {c->uL[0], c->uL[1], c->uL[2]}, {c->uR[0], c->uR[1], c->uR[2]},
                  {c->uadv[0], c->uadv[1], c->uadv[2]}, c->g, k});
    a7.push_back({{c->uadv[0], c->uadv[1], c->uadv[2]}, c->mrhs, c->g});
    a8.push_back({{c->uadv[0], c->uadv[1], c->uadv[2]}, c->phi_mac, {c->umac[0], c->umac[1], c->umac[2]}, c->g});
    a9.push_back({c->u, {c->uL[0], c->uL[1], c->uL[2]}, {c->uR[0], c->uR[1], c->uR[2]},
                  {c->umac[0], c->umac[1], c->umac[2]}, c->Gp, c->Lu, fo, c->rhs, c->g, k});
    a10.push_back({c->wn, c->nrhs, c->g, k});
    a12.push_back({c->p, c->ustar, c->Gp, c->wn, c->g, k});
    a11.push_back({c->ustar, c->Gp, c->p, c->g, k});
  }
  T.eta = table<OpEta<D>>(B, a1);
  T.ef = table<OpEtaFaces<D>>(B, a2);
  T.gp = table<OpGradP<D>>(B, a3);
  T.slopes = table<OpSlopes<D>>(B, a4);
  T.hats = table<OpHats<D>>(B, a5);
  T.traces = table<OpTraces<D>>(B, a6);
  T.macrhs = table<OpMacRhs<D>>(B, a7);
  T.maccorr = table<OpMacCorrect<D>>(B, a8);
  T.advect = table<OpAdvectRhs<D>>(B, a9);
  T.nrhs = table<OpNodalRhs<D>>(B, a10);
  T.gpw = table<OpGradPW<D>>(B, a12);
  T.update = table<OpProjectUpdate<D>>(B, a11);
}

struct BatchExplicit {
  ExplicitTables t;
};

void* explicit_create(hbf_batch* B) {
  auto* E = new BatchExplicit();
  if (B->dim == 2)
    build_tables<2>(B, E->t);
  else
    build_tables<3>(B, E->t);
  return E;
}

void explicit_destroy(void* p) { delete (BatchExplicit*)p; }

// Stages of Sec. III A-B: eta, face eta and G p; then (after the caller has
// launched L_eta u) slopes, transverse terms, face states and D^MAC u^adv.
template <int D>
static void pre_a(hbf_batch* B, BatchExplicit* E) {
  run<OpEta<D>>(B, E->t.eta, B->H[0][kCells], B->mask_all);
  run<OpEtaFaces<D>>(B, E->t.ef, B->H[0][kFaces], B->mask_all);
  run<OpGradP<D>>(B, E->t.gp, B->H[0][kCells], B->mask_all);
}

template <int D>
static void pre_b(hbf_batch* B, BatchExplicit* E) {
  run<OpSlopes<D>>(B, E->t.slopes, B->H[0][kCells], B->mask_all);
  run<OpHats<D>>(B, E->t.hats, B->H[0][kCells], B->mask_all);
  run<OpTraces<D>>(B, E->t.traces, B->H[0][kFaces], B->mask_all);
  run<OpMacRhs<D>>(B, E->t.macrhs, B->H[0][kCells], B->mask_all);
}

template <int D>
static void post(hbf_batch* B, BatchExplicit* E) {
  run<OpMacCorrect<D>>(B, E->t.maccorr, B->H[0][kFaces], B->mask_all);
  run<OpAdvectRhs<D>>(B, E->t.advect, B->H[0][kCells], B->mask_all);
}

template <int D>
static void nodal_rhs(hbf_batch* B, BatchExplicit* E) {
  run<OpGradPW<D>>(B, E->t.gpw, B->H[0][kCells], B->mask_all);
  run<OpNodalRhs<D>>(B, E->t.nrhs, B->H[0][kNodes], B->mask_all);
}

template <int D>
static void update(hbf_batch* B, BatchExplicit* E) {
  run<OpProjectUpdate<D>>(B, E->t.update, B->H[0][kCells], B->mask_all);
}

void explicit_stage(hbf_batch* B, void* e, int which) {
  auto* E = (BatchExplicit*)e;
  const bool d3 = B->dim == 3;
  switch (which) {
    case 0: d3 ? pre_a<3>(B, E) : pre_a<2>(B, E); break;
    case 1: d3 ? pre_b<3>(B, E) : pre_b<2>(B, E); break;
    case 2: d3 ? post<3>(B, E) : post<2>(B, E); break;
    case 3: d3 ? nodal_rhs<3>(B, E) : nodal_rhs<2>(B, E); break;
    case 4: d3 ? update<3>(B, E) : update<2>(B, E); break;
  }
}

}  // namespace batch
}  // namespace hb
