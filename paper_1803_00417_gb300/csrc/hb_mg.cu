// Multigrid solvers and reductions (host drivers + kernel instantiations).
//
// V(nu1, nu2) cycle, as stated for the three solves of Sec. III A:
//   nu1 smoothing sweeps; r = b - A x; restrict r to the next level's b;
//   x_coarse = 0; recurse; x += P x_coarse; nu2 sweeps.
//   coarsest level: nu_bottom sweeps in a single thread block.
//   stop when ||b - A x||_inf <= rtol ||b||_inf.
// Singular problems (MAC and nodal potentials) remove the (weighted) mean of
// the right-hand side and pin the mean of the iterate after each cycle and the
// bottom solve.
#include <cmath>
#include <cstdio>

#include "hb_internal.h"
#include "hb_mg_kernels.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// deterministic reductions: fixed grid, per-block partials, one final block
// ---------------------------------------------------------------------------
template <int MODE>  // 0: max |x| (non-finite -> +inf), 1: sum x, 2: weighted nodal sum
__global__ void k_reduce_partial(const double* __restrict__ x, long long n, double* __restrict__ part,
                                 Geom g, int dim) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double v = x[t];
    if (MODE == 0) {
      double a = fabs(v);
      if (!isfinite(a)) a = INFINITY;
      acc = fmax(acc, a);
    } else if (MODE == 1) {
      acc += v;
    } else {
      int e0 = g.n[0] + 1, e1 = g.n[1] + 1;
      int i = (int)(t % e0);
      int q = (int)(t / e0);
      int j = q % e1;
      int k = q / e1;
      double w = 1.0;
      if (i == 0 || i == g.n[0]) w *= 0.5;
      if (j == 0 || j == g.n[1]) w *= 0.5;
      if (dim == 3 && (k == 0 || k == g.n[2])) w *= 0.5;
      acc += w * v;
    }
  }
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = MODE == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = MODE == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

template <int MODE>
__global__ void k_reduce_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc = MODE == 0 ? fmax(acc, part[t]) : acc + part[t];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = MODE == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = MODE == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) *out = v;
  }
}

// x -= (*sum) * inv_count  (mean removal without a host round trip)
template <typename T>
__global__ void k_sub_mean(T* __restrict__ x, long long n, const double* __restrict__ sum, double inv_count) {
  T m = T(*sum * inv_count);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] -= m;
}

template <typename T>
__global__ void k_zero(T* __restrict__ x, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = T(0);
}

template <int MODE>
static int reduce_to_device(hbf_ctx* c, const double* x, long long n, double* out) {
  launch(c, kSlotNone, k_reduce_partial<MODE>, kRedBlocks, kThreads, x, n, c->partial, c->g, c->dim);
  launch(c, kSlotNone, k_reduce_final<MODE>, 1, 1024, c->partial, kRedBlocks, out);
  return cuda_check(c, cudaGetLastError(), "reduction");
}

static double read_result(hbf_ctx* c, const double* dev, int* st) {
  cudaError_t e = cudaMemcpyAsync(c->hres, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    *st = cuda_check(c, e, "reading a reduction");
    return NAN;
  }
  return *c->hres;
}

double reduce_max_abs(hbf_ctx* c, const double* x, long long n, int* st) {
  *st = reduce_to_device<0>(c, x, n, c->dres);
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

double reduce_sum(hbf_ctx* c, const double* x, long long n, int* st) {
  *st = reduce_to_device<1>(c, x, n, c->dres);
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

// ---------------------------------------------------------------------------
// problem interface for the generic driver
// ---------------------------------------------------------------------------
struct Problem {
  hbf_ctx* c;
  int nlev;
  bool singular;
  explicit Problem(hbf_ctx* ctx, bool sing) : c(ctx), nlev((int)ctx->lv.size()), singular(sing) {}
  virtual ~Problem() {}
  virtual double* x(int l) = 0;
  virtual double* b(int l) = 0;
  virtual double* r(int l) = 0;
  virtual long long count(int l) = 0;
  virtual void smooth(int l) = 0;
  virtual void resid(int l) = 0;
  virtual void restrict_to(int l) = 0;   // b(l+1) = R r(l)
  virtual void prolong_add(int l) = 0;   // x(l) += P x(l+1)
  virtual void bottom(int l) = 0;
  virtual int sub_mean(int l, double* v) { (void)l; (void)v; return 0; }
};

template <int D>
struct ViscProblem : Problem {
  double* x0;
  double beta;
  ViscProblem(hbf_ctx* ctx, double* x_in, double bt) : Problem(ctx, false), x0(x_in), beta(bt) {}
  double* x(int l) override { return l == 0 ? x0 : c->lv[l].vx; }
  double* b(int l) override { return c->lv[l].vb; }
  double* r(int l) override { return c->lv[l].vr; }
  long long count(int l) override { return (long long)D * c->lv[l].g.ncell; }
  void smooth(int l) override {
    const Level& L = c->lv[l];
    int nb = grid_for(rb_count<D>(L.g));
    for (int comp = 0; comp < D; ++comp)
      for (int col = 0; col < 2; ++col)
        launch(c, l == 0 ? kSlotViscSmooth : kSlotNone, k_visc_smooth<D, double>, nb, kThreads, x(l), L.vb, L.ef[0], L.ef[1], L.ef[2], L.g,
                                                                  comp, col, beta, l > 0);
  }
  void resid(int l) override {
    const Level& L = c->lv[l];
    launch(c, l == 0 ? kSlotViscResid : kSlotNone, k_visc_resid<D, double>, grid_for(L.g.ncell), kThreads, x(l), L.vb, L.vr, L.ef[0], L.ef[1],
                                                                             L.ef[2], L.g, beta, l > 0);
  }
  void restrict_to(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_restrict_cells<D, double>, grid_for((long long)D * C.g.ncell), kThreads, F.vr, C.vb, F.g,
                                                                                              C.g, D);
    launch(c, kSlotNone, k_zero<double>, grid_for((long long)D * C.g.ncell), kThreads, C.vx, (long long)D * C.g.ncell);
  }
  void prolong_add(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_prolong_cells_add<D, double>, grid_for((long long)D * F.g.ncell), kThreads, 
        x(l), C.vx, F.g, C.g, D, -1.0);
  }
  void bottom(int l) override {
    const Level& L = c->lv[l];
    launch(c, kSlotNone, k_visc_bottom<D, double>, 1, 1024, x(l), L.vb, L.ef[0], L.ef[1], L.ef[2], L.g, beta,
                                                         c->cfg.nu_bottom, l > 0);
  }
};

template <int D>
struct MacProblem : Problem {
  double* x0;
  MacProblem(hbf_ctx* ctx, double* x_in) : Problem(ctx, true), x0(x_in) {}
  double* x(int l) override { return l == 0 ? x0 : c->lv[l].cx; }
  double* b(int l) override { return c->lv[l].cb; }
  double* r(int l) override { return c->lv[l].cr; }
  long long count(int l) override { return c->lv[l].g.ncell; }
  void smooth(int l) override {
    const Level& L = c->lv[l];
    int nb = grid_for(rb_count<D>(L.g));
    for (int col = 0; col < 2; ++col)
      launch(c, l == 0 ? kSlotCellSmooth : kSlotNone, k_cell_smooth<D, double>, nb, kThreads, x(l), L.cb, L.g, col);
  }
  void resid(int l) override {
    const Level& L = c->lv[l];
    launch(c, l == 0 ? kSlotCellResid : kSlotNone, k_cell_resid<D, double>, grid_for(L.g.ncell), kThreads, x(l), L.cb, L.cr, L.g);
  }
  void restrict_to(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_restrict_cells<D, double>, grid_for(C.g.ncell), kThreads, F.cr, C.cb, F.g, C.g, 1);
    launch(c, kSlotNone, k_zero<double>, grid_for(C.g.ncell), kThreads, C.cx, C.g.ncell);
  }
  void prolong_add(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_prolong_cells_add<D, double>, grid_for(F.g.ncell), kThreads, x(l), C.cx, F.g, C.g, 1, 1.0);
  }
  void bottom(int l) override {
    const Level& L = c->lv[l];
    launch(c, kSlotNone, k_cell_bottom<D, double>, 1, 1024, x(l), L.cb, L.g, c->cfg.nu_bottom);
  }
  int sub_mean(int l, double* v) override {
    const Level& L = c->lv[l];
    int st = reduce_to_device<1>(c, v, L.g.ncell, c->dres + 1);
    if (st) return st;
    launch(c, kSlotNone, k_sub_mean<double>, grid_for(L.g.ncell), kThreads, v, L.g.ncell, c->dres + 1,
                                                                       1.0 / (double)L.g.ncell);
    return cuda_check(c, cudaGetLastError(), "k_sub_mean");
  }
};

template <int D>
struct NodalProblem : Problem {
  double* x0;
  NodalProblem(hbf_ctx* ctx, double* x_in) : Problem(ctx, true), x0(x_in) {}
  double* x(int l) override { return l == 0 ? x0 : c->lv[l].nx; }
  double* b(int l) override { return c->lv[l].nb; }
  double* r(int l) override { return c->lv[l].nr; }
  long long count(int l) override { return c->lv[l].g.nnode; }
  void smooth(int l) override {
    const Level& L = c->lv[l];
    for (int col = 0; col < (1 << D); ++col)
      launch(c, l == 0 ? kSlotNodalSmooth : kSlotNone, k_nodal_smooth<D, double>, grid_for(mc_count<D>(L.g, col)),
             kThreads, x(l), L.nb, L.g, col);
  }
  void resid(int l) override {
    const Level& L = c->lv[l];
    launch(c, l == 0 ? kSlotNodalResid : kSlotNone, k_nodal_resid<D, double>, grid_for(L.g.nnode), kThreads, x(l), L.nb, L.nr, L.g);
  }
  void restrict_to(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_restrict_nodes<D, double>, grid_for(C.g.nnode), kThreads, F.nr, C.nb, F.g, C.g);
    launch(c, kSlotNone, k_zero<double>, grid_for(C.g.nnode), kThreads, C.nx, C.g.nnode);
  }
  void prolong_add(int l) override {
    const Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotNone, k_prolong_nodes_add<D, double>, grid_for(F.g.nnode), kThreads, x(l), C.nx, F.g, C.g);
  }
  void bottom(int l) override {
    const Level& L = c->lv[l];
    launch(c, kSlotNone, k_nodal_bottom<D, double>, 1, 1024, x(l), L.nb, L.g, c->cfg.nu_bottom);
  }
  int sub_mean(int l, double* v) override {
    const Level& L = c->lv[l];
    Geom gsave = c->g;
    c->g = L.g;  // the weighted reduction reads the level geometry from the context
    int st = reduce_to_device<2>(c, v, L.g.nnode, c->dres + 1);
    c->g = gsave;
    if (st) return st;
    double wsum = (double)L.g.n[0] * L.g.n[1] * (D == 3 ? L.g.n[2] : 1);
    launch(c, kSlotNone, k_sub_mean<double>, grid_for(L.g.nnode), kThreads, v, L.g.nnode, c->dres + 1, 1.0 / wsum);
    return cuda_check(c, cudaGetLastError(), "k_sub_mean");
  }
};

static void vcycle(Problem& P, int l, const SolverCfg& cfg) {
  if (l == P.nlev - 1) {
    if (P.singular) P.sub_mean(l, P.b(l));
    P.bottom(l);
    if (P.singular) P.sub_mean(l, P.x(l));
    return;
  }
  for (int s = 0; s < cfg.nu1; ++s) P.smooth(l);
  P.resid(l);
  P.restrict_to(l);
  vcycle(P, l + 1, cfg);
  P.prolong_add(l);
  for (int s = 0; s < cfg.nu2; ++s) P.smooth(l);
}

static int mg_solve(Problem& P, const double* b_in, hbf_solve_stats* out) {
  hbf_ctx* c = P.c;
  const SolverCfg& cfg = c->cfg;
  long long n0 = P.count(0);
  int st = cuda_check(c, cudaMemcpyAsync(P.b(0), b_in, n0 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
                      "copy rhs");
  if (st) return st;
  if (P.singular) {
    if ((st = P.sub_mean(0, P.b(0)))) return st;
    if ((st = P.sub_mean(0, P.x(0)))) return st;
  }
  double bnorm = reduce_max_abs(c, P.b(0), n0, &st);
  if (st) return st;
  P.resid(0);
  double rn = reduce_max_abs(c, P.r(0), n0, &st);
  if (st) return st;
  double r0 = rn;
  if (bnorm == 0.0) bnorm = rn;
  double tol = cfg.rtol * bnorm;
  int cycles = 0;
  while (rn > tol && cycles < cfg.max_cycles && std::isfinite(rn)) {
    vcycle(P, 0, cfg);
    ++cycles;
    if (P.singular && (st = P.sub_mean(0, P.x(0)))) return st;
    P.resid(0);
    rn = reduce_max_abs(c, P.r(0), n0, &st);
    if (st) return st;
  }
  if ((st = cuda_check(c, cudaGetLastError(), "multigrid kernels"))) return st;
  hbf_solve_stats s;
  s.cycles = cycles;
  s.r0 = r0;
  s.rnorm = rn;
  s.bnorm = bnorm;
  s.converged = rn <= tol;
  if (out) *out = s;
  if (!std::isfinite(rn) || !std::isfinite(bnorm)) return fail(c, HBF_ERR_NONFINITE, "non-finite residual norm");
  if (!s.converged) {
    char buf[160];
    snprintf(buf, sizeof buf, "multigrid did not converge: %d cycles, residual %.3e > tol %.3e", cycles, rn, tol);
    return fail(c, HBF_ERR_NOT_CONVERGED, buf);
  }
  return HBF_OK;
}

// coarse-level face eta from the level-0 faces
template <int D>
static void build_eta_levels(hbf_ctx* c) {
  for (size_t l = 1; l < c->lv.size(); ++l) {
    const Level &F = c->lv[l - 1], &C = c->lv[l];
    for (int a = 0; a < D; ++a)
      launch(c, kSlotNone, k_restrict_faces<D, double>, grid_for(C.g.nface[a]), kThreads, F.ef[a], C.ef[a], a, F.g,
                                                                                       C.g);
  }
}

int solve_viscous(hbf_ctx* c, double beta, const double* rhs, double* u, hbf_solve_stats* s) {
  int st = launch_eta_faces(c);
  if (st) return st;
  if (c->dim == 2) {
    build_eta_levels<2>(c);
    ViscProblem<2> P(c, u, beta);
    return mg_solve(P, rhs, s);
  }
  build_eta_levels<3>(c);
  ViscProblem<3> P(c, u, beta);
  return mg_solve(P, rhs, s);
}

int solve_mac(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  if (c->dim == 2) {
    MacProblem<2> P(c, phi);
    return mg_solve(P, rhs, s);
  }
  MacProblem<3> P(c, phi);
  return mg_solve(P, rhs, s);
}

int solve_nodal(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  if (c->dim == 2) {
    NodalProblem<2> P(c, phi);
    return mg_solve(P, rhs, s);
  }
  NodalProblem<3> P(c, phi);
  return mg_solve(P, rhs, s);
}

}  // namespace hb
