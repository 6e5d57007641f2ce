// Start-up, steady state and cessation of the lid-driven cavity (Sec. III A:
// the steady criterion; Sec. IV: start-up from rest, the steady state, the
// lid stopped and the fluid brought to rest in finite time, yield surfaces,
// stagnant and plug zones; Sec. IV and V: centre-line profiles and vortex
// centres), plus the checkpoint record of a context.
//
// Diagnostics work on the context's current U:
//  * |tau| = 2 eta |gamma_dot| per cell (tau = 2 eta gamma_dot, the scaled
//    norm of Eq. 1), from the same strain rate and viscosity as stage 1;
//  * unyielded cells (|tau| <= tau_y) joined into zones through shared faces
//    by minimum-label propagation with pointer jumping (each cell's label
//    only decreases, and only its own thread writes it), then classified by
//    the walls they touch;
//  * the centre-line profile and the stream function of the centre plane
//    (one thread per node column summing up the column), and the node where
//    |psi| is largest (one block, ties to the smallest index).
// The drivers loop over hbf_step on the host and evaluate the criteria
// after every step.  This unit is compiled without FMA contraction, like the
// explicit stages, so that |gamma_dot| is the one stage 1 forms.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hb_explicit.cuh"
#include "hb_internal.h"

namespace hb {
namespace {

template <int D>
__global__ void k_tau_norm(const double* __restrict__ u, double* __restrict__ out, const __grid_constant__ Geom g,
                           Rheo r) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    const double gn = strain_norm_at<D>(u, g, t);
    out[t] = 2.0 * viscosity(gn, r) * gn;
  }
}

__global__ void k_absdiff(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                          long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = fabs(a[t] - b[t]);
}

__global__ void k_zone_init(const double* __restrict__ tau, double tau_y, int* __restrict__ lab,
                            int* __restrict__ touch, int n) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    lab[t] = tau[t] <= tau_y ? t : -1;
    touch[t] = 0;
  }
}

// one sweep of minimum-label propagation over face neighbours plus a
// pointer jump; *changed is set when any label decreased
template <int D>
__global__ void k_zone_step(int* __restrict__ lab, const __grid_constant__ Geom g, int* __restrict__ changed) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    const int l = lab[t];
    if (l < 0) continue;
    int i, j, k;
    cell_coords<D>(g, t, i, j, k);
    int m = l;
    const int p[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int stride = a == 0 ? 1 : (a == 1 ? g.n[0] : g.n[0] * g.n[1]);
      const int span = stride * g.n[a];  // a periodic axis wraps by one period
      if (p[a] > 0 || g.per[a]) {
        const int q = lab[p[a] > 0 ? t - stride : t - stride + span];
        if (q >= 0 && q < m) m = q;
      }
      if (p[a] < g.n[a] - 1 || g.per[a]) {
        const int q = lab[p[a] < g.n[a] - 1 ? t + stride : t + stride - span];
        if (q >= 0 && q < m) m = q;
      }
    }
    const int r = lab[m];  // m is a cell of the same zone, so r >= 0
    if (r < m) m = r;
    if (m < l) {
      lab[t] = m;
      *changed = 1;
    }
  }
}

// touch[root] |= 1 for a wall at rest, 2 for a moving wall, over the zone's
// cells next to a wall
template <int D>
__global__ void k_zone_touch(const int* __restrict__ lab, int* __restrict__ touch, const __grid_constant__ Geom g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    const int l = lab[t];
    if (l < 0) continue;
    int i, j, k;
    cell_coords<D>(g, t, i, j, k);
    const int p[3] = {i, j, k};
    int bits = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (g.per[a] || p[a] != (s ? g.n[a] - 1 : 0)) continue;
        const bool moving = g.wu[a][s][0] != 0.0 || g.wu[a][s][1] != 0.0 || g.wu[a][s][2] != 0.0;
        bits |= moving ? 2 : 1;
      }
    if (bits) atomicOr(&touch[l], bits);
  }
}

// cnt[0] yielded cells; cnt[1 + kind] unyielded cells and cnt[4 + kind] zones
// (roots) of kind 0 stagnant, 1 plug, 2 attached
__global__ void k_zone_count(const int* __restrict__ lab, const int* __restrict__ touch,
                             unsigned long long* __restrict__ cnt, int n) {
  __shared__ unsigned long long sc[7];
  if (threadIdx.x < 7) sc[threadIdx.x] = 0ull;
  __syncthreads();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int l = lab[t];
    if (l < 0) {
      atomicAdd(&sc[0], 1ull);
      continue;
    }
    const int tb = touch[l];
    const int kind = (tb & 1) ? 0 : ((tb & 2) ? 2 : 1);
    atomicAdd(&sc[1 + kind], 1ull);
    if (l == t) atomicAdd(&sc[4 + kind], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 7 && sc[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], sc[threadIdx.x]);
}

// u_x (comp c) of cell (i, j, k) averaged over the middle cells of the axes in
// `mask` (bit a: average across axis a), the higher axis innermost
template <int D>
__device__ double centre_avg(const double* __restrict__ uc, const Geom& g, int i, int j, int k, int mask) {
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  for (int a = 0; a < D; ++a)
    if (mask & (1 << a)) {
      hi[a] = g.n[a] / 2;
      lo[a] = (g.n[a] % 2 == 0) ? g.n[a] / 2 - 1 : g.n[a] / 2;
    }
  if (D == 2) {
    const int a = (mask & 1) ? 0 : 1;
    if (lo[a] == hi[a]) return uc[cidx<D>(g, lo[0], lo[1], 0)];
    return 0.5 * (uc[cidx<D>(g, lo[0], lo[1], 0)] + uc[cidx<D>(g, hi[0], hi[1], 0)]);
  }
  // 3D: average over the higher masked axis first, then the lower one
  int ax[2], na = 0;
  for (int a = 0; a < 3; ++a)
    if (mask & (1 << a)) ax[na++] = a;
  auto val = [&](int q0, int q1) {  // q0: choice along ax[0], q1 along ax[1] (0 lo, 1 hi)
    int p[3] = {i, j, k};
    p[ax[0]] = q0 ? hi[ax[0]] : lo[ax[0]];
    if (na > 1) p[ax[1]] = q1 ? hi[ax[1]] : lo[ax[1]];
    return uc[cidx<D>(g, p[0], p[1], p[2])];
  };
  if (na == 1) return lo[ax[0]] == hi[ax[0]] ? val(0, 0) : 0.5 * (val(0, 0) + val(1, 0));
  auto inner = [&](int q0) {
    return lo[ax[1]] == hi[ax[1]] ? val(q0, 0) : 0.5 * (val(q0, 0) + val(q0, 1));
  };
  return lo[ax[0]] == hi[ax[0]] ? inner(0) : 0.5 * (inner(0) + inner(1));
}

template <int D>
__global__ void k_centreline(const double* __restrict__ uc, int along, double* __restrict__ out,
                             const __grid_constant__ Geom g) {
  const int mask = ((1 << D) - 1) & ~(1 << along);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.n[along]; q += gridDim.x * blockDim.x) {
    int p[3] = {0, 0, 0};
    p[along] = q;
    out[q] = centre_avg<D>(uc, g, p[0], p[1], p[2], mask);
  }
}

// psi on the (na+1) x (nb+1) nodes of the centre plane; one thread per node
// column i sums h u_x over the cell rows
template <int D>
__global__ void k_psi(const double* __restrict__ ux, double* __restrict__ psi, const __grid_constant__ Geom g) {
  const int na = g.n[0], nb = D == 3 ? g.n[2] : g.n[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= na; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    psi[i] = 0.0;
    for (int j = 0; j < nb; ++j) {
      double face = 0.0;
      if (i > 0 && i < na) {
        const double a = D == 3 ? centre_avg<D>(ux, g, i - 1, 0, j, 2) : ux[cidx<D>(g, i - 1, j, 0)];
        const double b = D == 3 ? centre_avg<D>(ux, g, i, 0, j, 2) : ux[cidx<D>(g, i, j, 0)];
        face = 0.5 * (a + b);
      }
      acc += face;
      psi[i + (size_t)(na + 1) * (j + 1)] = g.h * acc;
    }
  }
}

// one block: the node of largest |psi| (smallest index among ties) and the
// values at it and its four in-plane neighbours (NaN where outside):
// res = {index, psi, psi(i-1), psi(i+1), psi(j-1), psi(j+1)}
__global__ void k_psi_peak(const double* __restrict__ psi, int ea, int eb, double* __restrict__ res) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  const int n = ea * eb;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double v = fabs(psi[t]);
    if (v > best || (v == best && t < bi)) {
      best = v;
      bi = t;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double v = sv[threadIdx.x + s];
      const int q = si[threadIdx.x + s];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && q < si[threadIdx.x])) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = q;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int k = si[0];
    const int i = k % ea, j = k / ea;
    res[0] = (double)k;
    res[1] = psi[k];
    res[2] = i > 0 ? psi[k - 1] : NAN;
    res[3] = i < ea - 1 ? psi[k + 1] : NAN;
    res[4] = j > 0 ? psi[k - ea] : NAN;
    res[5] = j < eb - 1 ? psi[k + ea] : NAN;
  }
}

int diag_scratch(hbf_ctx* c) {
  if (c->dscr) return HBF_OK;
  const long long n = (long long)c->g.ncell;
  const long long nd = (long long)c->dim * n;
  const long long npsi = (long long)(c->g.n[0] + 1) * ((c->dim == 3 ? c->g.n[2] : c->g.n[1]) + 1);
  void *a = nullptr, *b = nullptr, *q = nullptr;
  if (cudaMalloc(&a, sizeof(double) * (size_t)std::max(nd, npsi + 8)) != cudaSuccess ||
      cudaMalloc(&b, sizeof(int) * (size_t)(2 * n + 1)) != cudaSuccess ||
      cudaMalloc(&q, sizeof(unsigned long long) * 8) != cudaSuccess) {
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    cudaGetLastError();
    return fail(c, HBF_ERR_OOM, "diagnostics scratch");
  }
  c->allocs.push_back(a);
  c->allocs.push_back(b);
  c->allocs.push_back(q);
  c->dscr = (double*)a;
  c->dlab = (int*)b;
  c->dcnt = (unsigned long long*)q;
  return HBF_OK;
}

// |tau| of every cell into dscr; returns max |tau|
double tau_max(hbf_ctx* c, int* st) {
  if ((*st = diag_scratch(c))) return NAN;
  const int nb = grid_for(c->g.ncell);
  if (c->dim == 2)
    launch(c, kSlotNone, k_tau_norm<2>, nb, kThreads, (const double*)c->u, c->dscr, c->g, c->rheo);
  else
    launch(c, kSlotNone, k_tau_norm<3>, nb, kThreads, (const double*)c->u, c->dscr, c->g, c->rheo);
  if ((*st = cuda_check(c, cudaGetLastError(), "stress norm"))) return NAN;
  return reduce_max_abs(c, c->dscr, c->g.ncell, st);
}

int copy_out(hbf_ctx* c, void* dst, const void* src, size_t bytes) {
  int st = cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), "diagnostics copy");
  if (st) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "diagnostics");
}

}  // namespace
}  // namespace hb

using namespace hb;

extern "C" {

int hbf_get_state(hbf_ctx* c, hbf_state* s, double* u, double* p) {
  if (!c || !s) return HBF_ERR_ARG;
  std::memset(s, 0, sizeof *s);
  s->dim = c->dim;
  s->precision = c->precision;
  for (int a = 0; a < 3; ++a) s->n[a] = a < c->dim ? c->g.n[a] : 1;
  s->h = c->g.h;
  s->t = c->t;
  s->step = c->nstep;
  s->K = c->K;
  s->nexp = c->rheo.n;
  s->tau_y = c->rheo.tau;
  s->m = c->rheo.m;
  s->reg_power = c->rheo.reg_power;
  s->predictor_viscous = c->predictor_visc;
  s->theta = c->theta;
  for (int a = 0; a < 3; ++a) s->periodic[a] = c->g.per[a];
  s->rho = c->rho;
  for (int a = 0; a < 3; ++a) s->f[a] = c->f[a];
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 3; ++q) s->wall_u[(a * 2 + sd) * 3 + q] = c->g.wu[a][sd][q];
  int st = HBF_OK;
  if (u && (st = hbf_get_field(c, HBF_U, u))) return st;
  if (p && (st = hbf_get_field(c, HBF_P, p))) return st;
  return hbf_sync(c);
}

int hbf_set_state(hbf_ctx* c, const hbf_state* s, const double* u, const double* p) {
  if (!c || !s) return HBF_ERR_ARG;
  if (s->dim != c->dim || !(s->h == c->g.h)) return fail(c, HBF_ERR_ARG, "state of another grid");
  for (int a = 0; a < c->dim; ++a)
    if (s->n[a] != c->g.n[a]) return fail(c, HBF_ERR_ARG, "state of another grid");
  int st = hbf_set_rheology(c, s->K, s->nexp, s->tau_y, s->m, s->reg_power);
  if (st) return st;
  if ((st = hbf_set_density(c, s->rho))) return st;
  if ((st = hbf_set_body_force(c, s->f))) return st;
  if ((st = hbf_set_predictor_viscous(c, s->predictor_viscous))) return st;
  if ((st = hbf_set_theta(c, s->theta))) return st;
  const int per[3] = {s->periodic[0], s->periodic[1], s->periodic[2]};
  if ((st = hbf_set_periodic(c, per))) return st;
  if ((st = hbf_set_walls(c, s->wall_u))) return st;
  if (u && (st = hbf_set_field(c, HBF_U, u))) return st;
  if (p && (st = hbf_set_field(c, HBF_P, p))) return st;
  c->t = s->t;
  c->nstep = s->step;
  c->prev_valid = false;
  return hbf_sync(c);
}

int hbf_set_walls(hbf_ctx* c, const double wall_u[18]) {
  if (!c || !wall_u) return HBF_ERR_ARG;
  for (int a = 0; a < c->dim; ++a)
    if (wall_u[(a * 2 + 0) * 3 + a] != 0.0 || wall_u[(a * 2 + 1) * 3 + a] != 0.0)
      return fail(c, HBF_ERR_ARG, "a wall velocity has a normal component");
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 3; ++q)
        c->g.wu[a][sd][q] = (a < c->dim && q < c->dim && !c->g.per[a]) ? wall_u[(a * 2 + sd) * 3 + q] : 0.0;
  geom_finish(c->g);
  // the finest multigrid level carries the wall velocities (coarse levels
  // solve for homogeneous errors); the fused tail records are rebuilt in
  // case the tail starts on the finest level
  c->lv[0].g = c->g;
  c->tail_lf = -1;
  for (auto& k : c->tail_host)
    for (auto& h : k) h.clear();
  ++c->walls_version;
  return HBF_OK;
}

int hbf_step_change(hbf_ctx* c, double* change) {
  if (!c || !change) return HBF_ERR_ARG;
  if (!c->prev_valid) return fail(c, HBF_ERR_ARG, "no step since U was last set");
  int st = diag_scratch(c);
  if (st) return st;
  const long long n = (long long)c->dim * c->g.ncell;
  launch(c, kSlotNone, k_absdiff, grid_for(n), kThreads, (const double*)c->u, (const double*)c->ustar, c->dscr, n);
  if ((st = cuda_check(c, cudaGetLastError(), "step change"))) return st;
  const double du = reduce_max_abs(c, c->dscr, n, &st);
  if (st) return st;
  const double um = reduce_max_abs(c, c->ustar, n, &st);
  if (st) return st;
  *change = um > 0.0 ? du / um : INFINITY;
  return HBF_OK;
}

int hbf_yield(hbf_ctx* c, hbf_yield_info* info, int32_t* labels) {
  if (!c || !info) return HBF_ERR_ARG;
  std::memset(info, 0, sizeof *info);
  int st = 0;
  const double tm = tau_max(c, &st);
  if (st) return st;
  info->tau_max = tm;
  const int n = c->g.ncell;
  int* lab = c->dlab;
  int* touch = c->dlab + n;
  int* changed = c->dlab + 2 * n;
  const int nb = grid_for(n);
  launch(c, kSlotNone, k_zone_init, nb, kThreads, (const double*)c->dscr, c->rheo.tau, lab, touch, n);
  // propagate in batches of 8 sweeps until a batch changes nothing; a label
  // path is at most n cells long, so n + 8 sweeps always suffice
  int h_changed = 1;
  for (long long done = 0; h_changed && done <= (long long)n + 8; done += 8) {
    if ((st = cuda_check(c, cudaMemsetAsync(changed, 0, sizeof(int), c->stream), "zones"))) return st;
    for (int q = 0; q < 8; ++q) {
      if (c->dim == 2)
        launch(c, kSlotNone, k_zone_step<2>, nb, kThreads, lab, c->g, changed);
      else
        launch(c, kSlotNone, k_zone_step<3>, nb, kThreads, lab, c->g, changed);
    }
    if ((st = copy_out(c, &h_changed, changed, sizeof(int)))) return st;
  }
  if (h_changed) return fail(c, HBF_ERR_CUDA, "zone labels did not settle");
  if (c->dim == 2)
    launch(c, kSlotNone, k_zone_touch<2>, nb, kThreads, (const int*)lab, touch, c->g);
  else
    launch(c, kSlotNone, k_zone_touch<3>, nb, kThreads, (const int*)lab, touch, c->g);
  if ((st = cuda_check(c, cudaMemsetAsync(c->dcnt, 0, 8 * sizeof(unsigned long long), c->stream), "zones")))
    return st;
  launch(c, kSlotNone, k_zone_count, nb, kThreads, (const int*)lab, (const int*)touch, c->dcnt, n);
  unsigned long long h[8];
  if ((st = copy_out(c, h, c->dcnt, 8 * sizeof(unsigned long long)))) return st;
  info->yielded = (int64_t)h[0];
  for (int k = 0; k < 3; ++k) {
    info->cells[k] = (int64_t)h[1 + k];
    info->zones[k] = (int64_t)h[4 + k];
  }
  if (labels && (st = copy_out(c, labels, lab, sizeof(int) * (size_t)n))) return st;
  return cuda_check(c, cudaGetLastError(), "zones");
}

int hbf_run_steady(hbf_ctx* c, double dt, double tol, int64_t max_steps, hbf_run_info* info) {
  if (!c || !info || !(dt > 0.0) || !(tol > 0.0) || max_steps < 1) return HBF_ERR_ARG;
  std::memset(info, 0, sizeof *info);
  info->change = INFINITY;
  for (int64_t m = 1; m <= max_steps; ++m) {
    int st = hbf_step(c, dt, nullptr);
    if (st == HBF_ERR_NOT_CONVERGED)
      ++info->not_converged;
    else if (st)
      return st;
    double ch = 0.0;
    if ((st = hbf_step_change(c, &ch))) return st;
    info->steps = m;
    info->change = ch;
    if (ch < tol) {
      info->reached = 1;
      break;
    }
  }
  info->t = c->t;
  return HBF_OK;
}

int hbf_run_cessation(hbf_ctx* c, double dt, int64_t max_steps, int damp_steps, hbf_run_info* info) {
  if (!c || !info || !(dt > 0.0) || max_steps < 1 || damp_steps < 0) return HBF_ERR_ARG;
  if (!(c->rheo.tau > 0.0)) return fail(c, HBF_ERR_ARG, "cessation needs a yield stress");
  std::memset(info, 0, sizeof *info);
  const double rest[18] = {0};
  int st = hbf_set_walls(c, rest);
  if (st) return st;
  double prev = tau_max(c, &st) / c->rheo.tau;
  if (st) return st;
  info->tau_ratio = prev;
  info->t = c->t;
  info->t_c = info->t_c_interp = INFINITY;
  if (prev <= 1.0) {
    info->reached = 1;
    info->t_c = info->t_c_interp = 0.0;
    return HBF_OK;
  }
  const double t0 = c->t;
  const double theta = c->theta;
  for (int64_t m = 1; m <= max_steps; ++m) {
    c->theta = m <= damp_steps ? 1.0 : theta;  // backward Euler for the first damp_steps steps
    st = hbf_step(c, dt, nullptr);
    c->theta = theta;
    if (st == HBF_ERR_NOT_CONVERGED)
      ++info->not_converged;
    else if (st)
      return st;
    const double r = tau_max(c, &st) / c->rheo.tau;
    if (st) return st;
    info->steps = m;
    info->tau_ratio = r;
    if (r <= 1.0) {
      const double frac = prev > r ? (prev - 1.0) / (prev - r) : 1.0;
      info->reached = 1;
      info->t_c = c->t - t0;
      info->t_c_interp = (double)(m - 1) * dt + frac * dt;
      break;
    }
    prev = r;
  }
  info->t = c->t;
  return HBF_OK;
}

int hbf_centreline(hbf_ctx* c, int comp, int along, double* out) {
  if (!c || !out || comp < 0 || comp >= c->dim || along < 0 || along >= c->dim) return HBF_ERR_ARG;
  int st = diag_scratch(c);
  if (st) return st;
  const double* uc = c->u + (size_t)comp * c->g.ncell;
  const int n = c->g.n[along];
  if (c->dim == 2)
    launch(c, kSlotNone, k_centreline<2>, grid_for(n), kThreads, uc, along, c->dscr, c->g);
  else
    launch(c, kSlotNone, k_centreline<3>, grid_for(n), kThreads, uc, along, c->dscr, c->g);
  if ((st = cuda_check(c, cudaGetLastError(), "centre line"))) return st;
  return copy_out(c, out, c->dscr, sizeof(double) * (size_t)n);
}

int hbf_vortex(hbf_ctx* c, double* psi, double centre[2], double* psi_c) {
  if (!c || !centre || !psi_c) return HBF_ERR_ARG;
  int st = diag_scratch(c);
  if (st) return st;
  const int ea = c->g.n[0] + 1, eb = (c->dim == 3 ? c->g.n[2] : c->g.n[1]) + 1;
  const long long np = (long long)ea * eb;
  double* dpsi = c->dscr;
  double* dres = c->dscr + np;
  if (c->dim == 2)
    launch(c, kSlotNone, k_psi<2>, grid_for(ea), kThreads, (const double*)c->u, dpsi, c->g);
  else
    launch(c, kSlotNone, k_psi<3>, grid_for(ea), kThreads, (const double*)c->u, dpsi, c->g);
  launch(c, kSlotNone, k_psi_peak, 1, 1024, (const double*)dpsi, ea, eb, dres);
  if ((st = cuda_check(c, cudaGetLastError(), "stream function"))) return st;
  double r[6];
  if ((st = copy_out(c, r, dres, sizeof r))) return st;
  if (psi && (st = copy_out(c, psi, dpsi, sizeof(double) * (size_t)np))) return st;
  const int k = (int)r[0];
  const int idx[2] = {k % ea, k / ea};
  const double h = c->g.h;
  for (int a = 0; a < 2; ++a) {
    double x = idx[a] * h;
    const double fm = r[2 + 2 * a], fp = r[3 + 2 * a], f0 = r[1];
    if (!std::isnan(fm) && !std::isnan(fp)) {
      const double den = fm - 2.0 * f0 + fp;
      if (den != 0.0) x += 0.5 * h * (fm - fp) / den;
    }
    centre[a] = x;
  }
  *psi_c = r[1];
  return HBF_OK;
}

}  // extern "C"
