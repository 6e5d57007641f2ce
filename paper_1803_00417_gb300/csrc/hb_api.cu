// C-ABI entry points and the step orchestration (Sec. III A: one time step of
// the approximate projection method; the stage order follows the paper).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "hb_internal.h"

namespace hb {

int fail(hbf_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(hbf_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HBF_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? HBF_ERR_OOM : HBF_ERR_CUDA, m);
}

ProfRegion::ProfRegion(hbf_ctx* ctx, int s) : c(ctx), slot(s), on(prof_wants(ctx->prof, s)) {
  if (on) prof_mark(c, slot, true);
}
ProfRegion::~ProfRegion() {
  if (on) prof_mark(c, slot, false);
}

void prof_mark(hbf_ctx* c, int slot, bool start) {
  Prof& P = c->prof;
  if (P.used[slot] + 2 > P.ev[slot].size()) {
    if (P.ev[slot].size() >= 2 * kProfPairs) return;  // pool full: stop recording this slot
    size_t old = P.ev[slot].size();
    P.ev[slot].resize(old + 256);
    for (size_t q = old; q < P.ev[slot].size(); ++q) cudaEventCreate(&P.ev[slot][q]);
  }
  if (!start && (P.used[slot] & 1) == 0) return;  // unmatched stop (start was dropped)
  cudaEventRecord(P.ev[slot][P.used[slot]++], c->stream);
}

static void prof_release(hbf_ctx* c) {
  for (int s = 0; s < kSlotCount; ++s) {
    for (cudaEvent_t e : c->prof.ev[s]) cudaEventDestroy(e);
    c->prof.ev[s].clear();
    c->prof.used[s] = 0;
  }
}

static Geom make_geom(int dim, const int n[3], double h) {
  Geom g;
  std::memset(&g, 0, sizeof g);
  g.n[0] = n[0];
  g.n[1] = n[1];
  g.n[2] = dim == 3 ? n[2] : 1;
  g.h = h;
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  g.nnode = (g.n[0] + 1) * (g.n[1] + 1) * (dim == 3 ? g.n[2] + 1 : 1);
  g.nface[0] = (g.n[0] + 1) * g.n[1] * g.n[2];
  g.nface[1] = g.n[0] * (g.n[1] + 1) * g.n[2];
  g.nface[2] = dim == 3 ? g.n[0] * g.n[1] * (g.n[2] + 1) : 0;
  geom_finish(g);
  return g;
}

template <typename T>
static int alloc(hbf_ctx* c, T** p, long long count) {
  if (count <= 0) {
    *p = nullptr;
    return HBF_OK;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)count * sizeof(T));
  if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc");
  c->allocs.push_back(q);
  *p = (T*)q;
  return cudaMemsetAsync(q, 0, (size_t)count * sizeof(T), c->stream) == cudaSuccess ? HBF_OK
                                                                                     : fail(c, HBF_ERR_CUDA, "memset");
}

static bool can_coarsen(const Geom& g, int dim) {
  for (int a = 0; a < dim; ++a)
    if (g.n[a] % 2 != 0 || g.n[a] / 2 < 2) return false;
  return true;
}

static int allocate(hbf_ctx* c) {
  const Geom& g = c->g;
  const int D = c->dim;
  int st = 0;
#define A(ptr, cnt) \
  if ((st = alloc(c, &(ptr), (cnt)))) return st
  A(c->u, (long long)D * g.ncell);
  A(c->ustar, (long long)D * g.ncell);
  A(c->rhs, (long long)D * g.ncell);
  A(c->Gp, (long long)D * g.ncell);
  A(c->Lu, (long long)D * g.ncell);
  A(c->p, g.nnode);
  A(c->nrhs, g.nnode);
  A(c->nres0, g.nnode);
  A(c->eta, g.ncell);
  A(c->phi_mac, g.ncell);
  A(c->mrhs, g.ncell);
  A(c->slopes, (long long)D * D * g.ncell);
  A(c->hats, (long long)D * D * g.ncell);
  A(c->tcom, (long long)D * D * g.ncell);
  A(c->wn, (long long)D * g.ncell);
  for (int a = 0; a < D; ++a) {
    A(c->uL[a], (long long)D * g.nface[a]);
    A(c->uR[a], (long long)D * g.nface[a]);
    A(c->uadv[a], g.nface[a]);
    A(c->umac[a], g.nface[a]);
  }
  A(c->kb, (long long)D * g.ncell);
  A(c->kr, (long long)D * g.ncell);
  A(c->krh, (long long)D * g.ncell);
  A(c->kp, (long long)D * g.ncell);
  A(c->kv, (long long)D * g.ncell);
  A(c->ks, (long long)D * g.ncell);
  A(c->kt, (long long)D * g.ncell);
  A(c->kph, (long long)D * g.ncell);
  A(c->ksh, (long long)D * g.ncell);
  if (c->precision == HBF_MIXED) {
    A(c->fkr, (long long)D * g.ncell);
    A(c->fkrh, (long long)D * g.ncell);
    A(c->fkp, (long long)D * g.ncell);
    A(c->fkv, (long long)D * g.ncell);
    A(c->fks, (long long)D * g.ncell);
    A(c->fkt, (long long)D * g.ncell);
    A(c->fkph, (long long)D * g.ncell);
    A(c->fksh, (long long)D * g.ncell);
    A(c->fke, (long long)D * g.ncell);
  }
  for (int q = 0; q < 3; ++q) A(c->dense[q].Minv, (long long)(kDenseMax + 1) * (kDenseMax + 1));
  A(c->dX, (long long)kDenseMax * kDenseMax);
  A(c->dM, (long long)(kDenseMax + 1) * (kDenseMax + 1));
  A(c->dA, (long long)(kDenseMax + 1) * 2 * (kDenseMax + 1));
  A(c->partial, 2 * kRedBlocks);  // two-result reductions use both halves
  A(c->dres, 8);
  A(c->sweep_err, 1);
  if (cudaMallocHost((void**)&c->hres, 8 * sizeof(double)) != cudaSuccess)
    return fail(c, HBF_ERR_OOM, "cudaMallocHost");
  // multigrid hierarchy
  Geom gl = g;
  for (int l = 0;; ++l) {
    Level L;
    L.g = gl;
    if (l > 0 || c->precision == HBF_MIXED) {
      A(L.vx, (long long)D * gl.ncell);
      A(L.cx, gl.ncell);
      A(L.nx, gl.nnode);
    }
    if (c->precision == HBF_MIXED) {
      A(L.fvx, (long long)D * gl.ncell);
      A(L.fvb, (long long)D * gl.ncell);
      A(L.fvr, (long long)D * gl.ncell);
      A(L.fcx, gl.ncell);
      A(L.fcb, gl.ncell);
      A(L.fcr, gl.ncell);
      A(L.fnx, gl.nnode);
      A(L.fnb, gl.nnode);
      A(L.fnr, gl.nnode);
      for (int a = 0; a < D; ++a) A(L.fef[a], gl.nface[a]);
      if (l == 0) A(L.feta, gl.ncell);
      if (l == 0 && D == 3) A(L.fvx2, (long long)D * gl.ncell);
    }
    A(L.vb, (long long)D * gl.ncell);
    A(L.vr, (long long)D * gl.ncell);
    A(L.cb, gl.ncell);
    A(L.cr, gl.ncell);
    A(L.nb, gl.nnode);
    A(L.nr, gl.nnode);
    for (int a = 0; a < D; ++a) A(L.ef[a], gl.nface[a]);
    c->lv.push_back(L);
    if (!can_coarsen(gl, D)) break;
    gl = D == 3 ? coarse_of<3>(gl) : coarse_of<2>(gl);
  }
#undef A
  return cuda_check(c, cudaStreamSynchronize(c->stream), "allocation");
}

struct FieldView {
  double* ptr[3];
  long long cnt[3];
  int parts;
};

static int field_view(hbf_ctx* c, int which, FieldView* v) {
  const Geom& g = c->g;
  const int D = c->dim;
  v->parts = 1;
  switch (which) {
    case HBF_U: v->ptr[0] = c->u; v->cnt[0] = (long long)D * g.ncell; return 0;
    case HBF_P: v->ptr[0] = c->p; v->cnt[0] = g.nnode; return 0;
    case HBF_ETA: v->ptr[0] = c->eta; v->cnt[0] = g.ncell; return 0;
    case HBF_USTAR: v->ptr[0] = c->ustar; v->cnt[0] = (long long)D * g.ncell; return 0;
    case HBF_RHS: v->ptr[0] = c->rhs; v->cnt[0] = (long long)D * g.ncell; return 0;
    case HBF_PHI_MAC: v->ptr[0] = c->phi_mac; v->cnt[0] = g.ncell; return 0;
    case HBF_GP: v->ptr[0] = c->Gp; v->cnt[0] = (long long)D * g.ncell; return 0;
    case HBF_LU: v->ptr[0] = c->Lu; v->cnt[0] = (long long)D * g.ncell; return 0;
    case HBF_SLOPES: v->ptr[0] = c->slopes; v->cnt[0] = (long long)D * D * g.ncell; return 0;
    case HBF_HATS: v->ptr[0] = c->hats; v->cnt[0] = (long long)D * D * g.ncell; return 0;
    case HBF_NRES0: v->ptr[0] = c->nres0; v->cnt[0] = g.nnode; return 0;
    case HBF_VRES0:
    case HBF_VCORR:
      if (!c->vres0) return -1;
      v->ptr[0] = which == HBF_VRES0 ? c->vres0 : c->vcorr;
      v->cnt[0] = (long long)D * g.ncell;
      return 0;
    case HBF_ETA_FACES:
      v->parts = D;
      for (int a = 0; a < D; ++a) {
        v->ptr[a] = c->lv[0].ef[a];
        v->cnt[a] = g.nface[a];
      }
      return 0;
    case HBF_UADV:
    case HBF_UMAC:
    case HBF_UL:
    case HBF_UR:
      v->parts = D;
      for (int a = 0; a < D; ++a) {
        double* src = which == HBF_UADV ? c->uadv[a] : which == HBF_UMAC ? c->umac[a]
                      : which == HBF_UL ? c->uL[a] : c->uR[a];
        v->ptr[a] = src;
        v->cnt[a] = (which == HBF_UL || which == HBF_UR) ? (long long)D * g.nface[a] : g.nface[a];
      }
      return 0;
  }
  return -1;
}

}  // namespace hb

using namespace hb;

extern "C" {

int hbf_init_grid(hbf_ctx** out, int dim, const int64_t n[3], double h, const double wall_u[18], int precision,
                  void* stream) {
  if (!out) return HBF_ERR_ARG;
  *out = nullptr;
  if (dim != 2 && dim != 3) return HBF_ERR_ARG;
  if (!(h > 0.0) || !n) return HBF_ERR_ARG;
  if (precision != HBF_FP64 && precision != HBF_MIXED) return HBF_ERR_ARG;
  int ni[3] = {1, 1, 1};
  long long tot = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 2 || n[a] > (1 << 20)) return HBF_ERR_ARG;
    ni[a] = (int)n[a];
    tot *= (n[a] + 1);
  }
  if (tot * dim >= (1LL << 31)) return HBF_ERR_ARG;
  hbf_ctx* c = new (std::nothrow) hbf_ctx();
  if (!c) return HBF_ERR_OOM;
  c->dim = dim;
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->g = make_geom(dim, ni, h);
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 3; ++q) c->g.wu[a][s][q] = 0.0;
  if (wall_u) {
    for (int a = 0; a < dim; ++a)
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < dim; ++q) c->g.wu[a][s][q] = wall_u[(a * 2 + s) * 3 + q];
    for (int a = 0; a < dim; ++a)
      if (c->g.wu[a][0][a] != 0.0 || c->g.wu[a][1][a] != 0.0) {
        delete c;
        return HBF_ERR_ARG;
      }
  }
  geom_finish(c->g);  // again: the FP32 copies of the wall velocities
  c->rheo.c2 = 1.0;
  c->rheo.n = 1.0;
  c->rheo.tau = 0.0;
  c->rheo.m = 1e4;
  c->rheo.reg_power = 1;
  c->rheo.e2 = rheo_e2(1.0, 1);
  int st = allocate(c);
  if (st) {
    hbf_destroy(c);
    return st;
  }
  *out = c;
  return HBF_OK;
}

void hbf_destroy(hbf_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  release_guess(c);
  release_visc_guess(c);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hres) cudaFreeHost(c->hres);
  prof_release(c);
  delete c;
}

int hbf_profile_enable(hbf_ctx* c, int on) {
  if (!c) return HBF_ERR_ARG;
  int st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
  if (st) return st;
  for (int s = 0; s < kSlotCount; ++s) c->prof.used[s] = 0;
  c->prof.level = on < 0 ? 0 : (on > 2 ? 2 : on);
  return HBF_OK;
}

int hbf_profile_read(hbf_ctx* c, int slot, double* total_ms, int64_t* launches) {
  if (!c || slot < 0 || slot >= kSlotCount || !total_ms || !launches) return HBF_ERR_ARG;
  int st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
  if (st) return st;
  double tot = 0.0;
  size_t pairs = c->prof.used[slot] / 2;
  for (size_t q = 0; q < pairs; ++q) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, c->prof.ev[slot][2 * q], c->prof.ev[slot][2 * q + 1]);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaEventElapsedTime");
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int64_t)pairs;
  return HBF_OK;
}

int64_t hbf_launch_count(const hbf_ctx* c) { return c ? (int64_t)c->nlaunch : HBF_ERR_ARG; }

const char* hbf_last_error(const hbf_ctx* c) { return c ? c->err.c_str() : "null context"; }

int hbf_sync(hbf_ctx* c) {
  if (!c) return HBF_ERR_ARG;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "hbf_sync");
}

int hbf_set_rheology(hbf_ctx* c, double K, double n, double tau_y, double m, int reg_power) {
  if (!c) return HBF_ERR_ARG;
  if (!(K >= 0.0) || !(n > 0.0) || !(tau_y >= 0.0) || !(m > 0.0)) return fail(c, HBF_ERR_ARG, "bad rheology");
  if (!reg_power && n < 1.0) return fail(c, HBF_ERR_ARG, "reg_power = 0 needs n >= 1 (eta bounded at g = 0)");
  c->K = K;
  c->rheo.c2 = std::pow(2.0, n - 1.0) * K;
  c->rheo.n = n;
  c->rheo.tau = tau_y;
  c->rheo.m = m;
  c->rheo.reg_power = reg_power ? 1 : 0;
  c->rheo.e2 = rheo_e2(n, c->rheo.reg_power);
  return HBF_OK;
}

int hbf_set_density(hbf_ctx* c, double rho) {
  if (!c) return HBF_ERR_ARG;
  if (!(rho > 0.0)) return fail(c, HBF_ERR_ARG, "rho must be positive");
  c->rho = rho;
  return HBF_OK;
}

int hbf_set_body_force(hbf_ctx* c, const double f[3]) {
  if (!c || !f) return HBF_ERR_ARG;
  for (int a = 0; a < 3; ++a) c->f[a] = a < c->dim ? f[a] : 0.0;
  return HBF_OK;
}

int hbf_set_theta(hbf_ctx* c, double theta) {
  if (!c) return HBF_ERR_ARG;
  if (!(theta >= 0.5 && theta <= 1.0)) return fail(c, HBF_ERR_ARG, "theta must lie in [1/2, 1]");
  c->theta = theta;
  return HBF_OK;
}

int hbf_set_predictor_viscous(hbf_ctx* c, int on) {
  if (!c) return HBF_ERR_ARG;
  c->predictor_visc = on ? 1 : 0;
  return HBF_OK;
}

int hbf_set_solver(hbf_ctx* c, double rtol, int max_cycles, int nu1, int nu2, int nu_bottom) {
  if (!c) return HBF_ERR_ARG;
  if (!(rtol > 0.0) || max_cycles < 1 || nu1 < 0 || nu2 < 0 || nu_bottom < 1)
    return fail(c, HBF_ERR_ARG, "bad solver settings");
  c->cfg.rtol = rtol;
  c->cfg.max_cycles = max_cycles;
  c->cfg.nu1 = nu1;
  c->cfg.nu2 = nu2;
  c->cfg.nu_bottom = nu_bottom;
  return HBF_OK;
}

int hbf_set_inner_drop(hbf_ctx* c, double drop) {
  if (!c) return HBF_ERR_ARG;
  if (!(drop >= 1e-7 && drop < 1.0)) return fail(c, HBF_ERR_ARG, "inner drop outside [1e-7, 1)");
  c->inner_drop = drop;
  return HBF_OK;
}

int hbf_set_split_layout(hbf_ctx* c, int on) {
  if (!c) return HBF_ERR_ARG;
  if (on != 0 && on != 1) return fail(c, HBF_ERR_ARG, "split layout must be 0 or 1");
  c->split_layout = on;
  return HBF_OK;
}

int hbf_set_periodic(hbf_ctx* c, const int periodic[3]) {
  if (!c || !periodic) return HBF_ERR_ARG;
  int per[3] = {0, 0, 0};
  for (int a = 0; a < c->dim; ++a) {
    per[a] = periodic[a] ? 1 : 0;
    if (per[a] && (c->g.n[a] % 2 != 0 || c->g.n[a] < 2))
      return fail(c, HBF_ERR_ARG, "a periodic axis needs an even cell count");
  }
  for (int a = 0; a < 3; ++a) {
    c->g.per[a] = per[a];
    if (per[a])  // no walls normal to a periodic axis
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < 3; ++q) c->g.wu[a][s][q] = 0.0;
  }
  geom_finish(c->g);
  c->lv[0].g = c->g;
  for (size_t l = 1; l < c->lv.size(); ++l)
    for (int a = 0; a < 3; ++a) c->lv[l].g.per[a] = per[a];
  // operators changed: rebuild the exact bottom inverses and the tail records
  for (auto& d : c->dense) d.valid = false;
  c->tail_lf = -1;
  for (auto& k : c->tail_host)
    for (auto& h : k) h.clear();
  ++c->walls_version;
  return HBF_OK;
}

int hbf_set_visc_guess(hbf_ctx* c, int mode) {
  if (!c) return HBF_ERR_ARG;
  if (mode < 0 || mode > 2) return fail(c, HBF_ERR_ARG, "viscous guess mode must be 0, 1 or 2");
  if (mode > 0 && c->precision != HBF_MIXED) return fail(c, HBF_ERR_ARG, "the viscous guess needs a mixed context");
  if (mode > 0 && !c->vprev32) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(float) * (size_t)c->dim * c->g.ncell) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HBF_ERR_OOM, "viscous guess buffer");
    }
    c->allocs.push_back(q);
    c->vprev32 = (float*)q;
  }
  c->vguess_mode = mode;
  c->vprev_ok = false;
  return HBF_OK;
}

int hbf_set_visc_record(hbf_ctx* c, int on) {
  if (!c) return HBF_ERR_ARG;
  if (on && c->precision != HBF_MIXED) return fail(c, HBF_ERR_ARG, "recording needs a mixed context");
  if (on && !c->vres0) {
    void *a = nullptr, *b = nullptr;
    const size_t bytes = sizeof(double) * (size_t)c->dim * c->g.ncell;
    if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess) {
      if (a) cudaFree(a);
      cudaGetLastError();
      return fail(c, HBF_ERR_OOM, "recording buffers");
    }
    c->allocs.push_back(a);
    c->allocs.push_back(b);
    c->vres0 = (double*)a;
    c->vcorr = (double*)b;
  }
  c->vrecord = on ? 1 : 0;
  return HBF_OK;
}

int hbf_restrict(hbf_ctx* c, int kind, int level, const double* src, double* dst) {
  if (!c || !src || !dst || kind < 0 || kind > 2) return HBF_ERR_ARG;
  if (level < 0 || level + 1 >= (int)c->lv.size()) return fail(c, HBF_ERR_ARG, "no coarser level");
  if (kind == 2)
    nodal_restrict(c, level, src, dst);
  else
    cell_restrict_d(c, level, src, dst, kind == 0 ? c->dim : 1);
  return cuda_check(c, cudaGetLastError(), "restriction");
}

int hbf_set_fused_sweep(hbf_ctx* c, int on) {
  if (!c) return HBF_ERR_ARG;
  c->fused_sweep = on ? 1 : 0;
  return HBF_OK;
}

int hbf_set_staged_sweep(hbf_ctx* c, int tile_x, int tile_z) {
  if (!c) return HBF_ERR_ARG;
  if ((tile_x != 0 && tile_x != 64 && tile_x != 128) || tile_z < 1 || tile_z > 4096)
    return fail(c, HBF_ERR_ARG, "staged sweep tile: width 0, 64 or 128, 1 <= planes <= 4096");
  c->staged_tx = tile_x;
  c->staged_tz = tile_z;
  return HBF_OK;
}

int hbf_set_staged_op(hbf_ctx* c, int rows, int tile_z) {
  if (!c) return HBF_ERR_ARG;
  if ((rows != 0 && rows != 4 && rows != 8) || tile_z < 1 || tile_z > 4096)
    return fail(c, HBF_ERR_ARG, "staged operator tile: rows 0, 4 or 8, 1 <= planes <= 4096");
  c->staged_op_rows = rows;
  c->staged_op_tz = tile_z;
  return HBF_OK;
}

int hbf_set_tail(hbf_ctx* c, int max_cells) {
  if (!c) return HBF_ERR_ARG;
  if (max_cells < 0) return fail(c, HBF_ERR_ARG, "negative tail size");
  if (max_cells != c->tail_cells) {
    c->tail_cells = max_cells;
    c->tail_lf = -1;  // recomputed, and the tail records rebuilt, at the next cycle
    for (auto& k : c->tail_host)
      for (auto& h : k) h.clear();
  }
  return HBF_OK;
}

int64_t hbf_field_size(const hbf_ctx* c, int which) {
  if (!c) return HBF_ERR_ARG;
  FieldView v;
  if (field_view(const_cast<hbf_ctx*>(c), which, &v)) return HBF_ERR_ARG;
  int64_t s = 0;
  for (int q = 0; q < v.parts; ++q) s += v.cnt[q];
  return s;
}

static int copy_field(hbf_ctx* c, int which, double* host_or_dev, bool in) {
  if (!c || !host_or_dev) return HBF_ERR_ARG;
  FieldView v;
  if (field_view(c, which, &v)) return fail(c, HBF_ERR_ARG, "unknown field");
  long long off = 0;
  for (int q = 0; q < v.parts; ++q) {
    size_t bytes = (size_t)v.cnt[q] * sizeof(double);
    cudaError_t e = in ? cudaMemcpyAsync(v.ptr[q], host_or_dev + off, bytes, cudaMemcpyDefault, c->stream)
                       : cudaMemcpyAsync(host_or_dev + off, v.ptr[q], bytes, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "field copy");
    off += v.cnt[q];
  }
  return HBF_OK;
}

int hbf_set_field(hbf_ctx* c, int which, const double* src) {
  if (c && (which == HBF_U || which == HBF_USTAR)) {
    c->prev_valid = false;
    c->vprev_ok = false;
  }
  return copy_field(c, which, const_cast<double*>(src), true);
}

int hbf_get_field(hbf_ctx* c, int which, double* dst) { return copy_field(c, which, dst, false); }

int hbf_compute_viscosity(hbf_ctx* c) {
  if (!c) return HBF_ERR_ARG;
  return launch_eta(c);
}

int hbf_predict(hbf_ctx* c, double dt) {
  if (!c) return HBF_ERR_ARG;
  if (!(dt > 0.0)) return fail(c, HBF_ERR_ARG, "dt must be positive");
  return launch_predict(c, dt);
}

int hbf_mac_project(hbf_ctx* c, hbf_solve_stats* s) {
  if (!c) return HBF_ERR_ARG;
  int st = launch_mac_rhs(c, c->mrhs);
  if (st) return st;
  if ((st = cuda_check(c, cudaMemsetAsync(c->phi_mac, 0, (size_t)c->g.ncell * sizeof(double), c->stream),
                       "memset phi")))
    return st;
  int sst = solve_mac(c, c->mrhs, c->phi_mac, s);
  if (sst && sst != HBF_ERR_NOT_CONVERGED) return sst;
  st = launch_mac_correct(c, c->phi_mac);
  return st ? st : sst;
}

int hbf_advect_rhs(hbf_ctx* c, double dt) {
  if (!c) return HBF_ERR_ARG;
  if (!(dt > 0.0)) return fail(c, HBF_ERR_ARG, "dt must be positive");
  return launch_advect_rhs(c, dt);
}

int hbf_solve_viscous(hbf_ctx* c, double dt, const double* rhs_dev, double* u_dev, hbf_solve_stats* s) {
  if (!c || !rhs_dev || !u_dev) return HBF_ERR_ARG;
  if (!(dt > 0.0)) return fail(c, HBF_ERR_ARG, "dt must be positive");
  return solve_viscous(c, visc_beta(dt, c->rho, c->theta), rhs_dev, u_dev, s);
}

int hbf_project(hbf_ctx* c, double dt, double* u_dev, double* p_dev, hbf_solve_stats* s) {
  if (!c || !u_dev || !p_dev) return HBF_ERR_ARG;
  if (!(dt > 0.0)) return fail(c, HBF_ERR_ARG, "dt must be positive");
  int st = launch_nodal_rhs(c, dt, u_dev, p_dev, c->nrhs);
  if (st) return st;
  if ((st = nodal_residual(c, c->nrhs, p_dev, c->nres0))) return st;
  int used = 0;
  if (c->guess && (st = apply_guess(c, c->nrhs, p_dev, &used))) return st;
  int sst = solve_nodal(c, c->nrhs, p_dev, s);
  if (s) s->guess = used;
  if (sst && sst != HBF_ERR_NOT_CONVERGED) return sst;
  st = launch_project_update(c, dt, u_dev, nullptr, p_dev);
  return st ? st : sst;
}

int hbf_step(hbf_ctx* c, double dt, hbf_step_stats* stats) {
  if (!c) return HBF_ERR_ARG;
  if (!(dt > 0.0)) return fail(c, HBF_ERR_ARG, "dt must be positive");
  hbf_step_stats local;
  hbf_step_stats* s = stats ? stats : &local;
  std::memset(s, 0, sizeof *s);
  int worst = HBF_OK;
  int st;
  if ((st = launch_eta(c))) return st;
  if ((st = launch_predict(c, dt))) return st;
  st = hbf_mac_project(c, &s->mac);
  if (st && st != HBF_ERR_NOT_CONVERGED) return st;
  if (st) worst = st;
  if ((st = launch_advect_rhs(c, dt))) return st;
  if ((st = cuda_check(c, cudaMemcpyAsync(c->ustar, c->u, (size_t)c->dim * c->g.ncell * sizeof(double),
                                          cudaMemcpyDeviceToDevice, c->stream),
                       "guess copy")))
    return st;
  st = solve_viscous(c, visc_beta(dt, c->rho, c->theta), c->rhs, c->ustar, &s->visc);
  if (st && st != HBF_ERR_NOT_CONVERGED) return st;
  if (st) worst = st;
  if ((c->vguess_mode > 0 || c->vrecord) && (st = visc_after_solve(c, c->ustar, c->u))) return st;
  st = hbf_project(c, dt, c->ustar, c->p, &s->nodal);
  if (st && st != HBF_ERR_NOT_CONVERGED) return st;
  if (st) worst = st;
  double* t = c->u;
  c->u = c->ustar;
  c->ustar = t;  // now u^m, which hbf_step_change compares with
  c->prev_valid = true;
  c->t += dt;
  ++c->nstep;
  return worst;
}

double hbf_cfl_dt(hbf_ctx* c, double cfl) {
  if (!c) return NAN;
  int st = 0;
  double umax = reduce_max_abs(c, c->u, (long long)c->dim * c->g.ncell, &st);
  if (st) return NAN;
  if (!std::isfinite(umax)) {  // the reduction maps NaN and Inf to +inf
    fail(c, HBF_ERR_NONFINITE, "non-finite velocity");
    return NAN;
  }
  return cfl * c->g.h / std::fmax(umax, 1.0);
}

}  // extern "C"
