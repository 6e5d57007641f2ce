// Batched sweep: many independent cavities of different sizes advanced by one
// time step each (Sec. III A), every stage one persistent launch over a tile
// work list spanning all cavities.  The multigrid cycles of all cavities run
// level by level together (a cavity whose hierarchy is shallower takes its
// exact bottom solve in the single batched bottom launch); the Krylov and
// defect-correction loops keep one state per cavity on the host, and a cavity
// that has converged is masked out of every later launch.  Fixed launch
// sequences (explicit stages, V-cycles) are captured once as CUDA graphs.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include "hb_batch_internal.h"
#include "hb_mg_kernels.cuh"
#include "hb_vcycle_tail.cuh"

namespace hb {
namespace batch {

// ---------------------------------------------------------------------------
// per-element operations (device)
// ---------------------------------------------------------------------------
template <int D, typename T, int C>
struct OpViscSmooth {
  using Arg = ViscArg<T>;
  static __device__ void apply(const Arg& a, int t, int col) {
    k_visc_smooth_c_at<D, T, C, false>(a.x, a.b, a.ef[0], a.ef[1], a.ef[2], a.g, col, a.beta, a.hom, t);
  }
};

// out = b - (x - beta L x), or x - beta L x when b is null
template <int D, typename T>
struct OpViscOp {
  using Arg = ViscArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    k_visc_op_at<D, T, false>(a.x, a.b, a.out, a.ef[0], a.ef[1], a.ef[2], a.g, a.beta, a.hom, t);
  }
};

// out = L_eta x (inhomogeneous walls), the predictor's stress term
template <int D>
struct OpTensorLu {
  using Arg = ViscArg<double>;
  static __device__ void apply(const Arg& a, int t, int) {
    k_tensor_lu_at<D, double>(a.x, a.out, a.ef[0], a.ef[1], a.ef[2], a.g, 0, t);
  }
};

template <int D, typename T>
struct OpCellSmooth {
  using Arg = PoisArg<T>;
  static __device__ void apply(const Arg& a, int t, int col) { k_cell_smooth_at<D, T, false>(a.x, a.b, a.g, col, t); }
};

template <int D, typename T>
struct OpCellResid {
  using Arg = PoisArg<T>;
  static __device__ void apply(const Arg& a, int t, int) { k_cell_resid_at<D, T, false>(a.x, a.b, a.r, a.g, t); }
};

template <int D, typename T>
struct OpNodalSmooth {
  using Arg = PoisArg<T>;
  static __device__ void apply(const Arg& a, int t, int col) { k_nodal_smooth_at<D, T, false>(a.x, a.b, a.g, col, t); }
};

template <int D, typename T>
struct OpNodalResid {
  using Arg = PoisArg<T>;
  static __device__ void apply(const Arg& a, int t, int) { k_nodal_resid_at<D, T, false>(a.x, a.b, a.r, a.g, t); }
};

template <int D, typename T>
struct OpRestrictCells {
  using Arg = XferArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    k_restrict_cells_at<D, T>(a.src, a.dst, a.gf, a.gc, a.ncomp, t);
    a.zero[t] = T(0);
  }
};

template <int D, typename T>
struct OpProlongCells {
  using Arg = XferArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    k_prolong_cells_add_at<D, T, false>(a.dst, a.src, a.gf, a.gc, a.ncomp, T(a.sign), t);
  }
};

template <int D, typename T>
struct OpRestrictNodes {
  using Arg = XferArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    k_restrict_nodes_at<D, T, false>(a.src, a.dst, a.gf, a.gc, t);
    a.zero[t] = T(0);
  }
};

template <int D, typename T>
struct OpProlongNodes {
  using Arg = XferArg<T>;
  static __device__ void apply(const Arg& a, int t, int) { k_prolong_nodes_add_at<D, T>(a.dst, a.src, a.gf, a.gc, t); }
};

// coarse face viscosity (mean of the fine faces it covers) and FP32 copies
struct FaceArg {
  const double* src[3];
  double* dst[3];
  float* fdst[3];
  Geom gf, gc;
};

template <int D>
struct OpRestrictFaces {
  using Arg = FaceArg;
  static __device__ void apply(const Arg& a, int t, int) {
    const int ax = face_axis(a.gc, t);
    k_restrict_faces_at<D, double>(a.src[ax], a.dst[ax], ax, a.gf, a.gc, t);
  }
};

struct OpFacesF32 {
  using Arg = FaceArg;
  static __device__ void apply(const Arg& a, int t, int) {
    const int ax = face_axis(a.gf, t);
    a.fdst[ax][t] = (float)a.src[ax][t];
  }
};

// vector updates; s points at the cavity's scalars:
// s[0] = beta, s[1] = omega (direction update), s[2] = alpha, s[3] = omega
template <typename T>
struct VecArg {
  T* x;
  const T* y;
  const T* z;
  const double* s;
};

template <typename T>
struct OpCopy {
  using Arg = VecArg<T>;
  static __device__ void apply(const Arg& a, int t, int) { a.x[t] = a.y[t]; }
};

template <typename T>
struct OpZero {
  using Arg = VecArg<T>;
  static __device__ void apply(const Arg& a, int t, int) { a.x[t] = T(0); }
};

// p = r + beta (p - omega v)
template <typename T>
struct OpBicgP {
  using Arg = VecArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    const T beta = (T)a.s[0], omega = (T)a.s[1];
    a.x[t] = a.y[t] + beta * (a.x[t] - omega * a.z[t]);
  }
};

// out = y - s[j] z
template <typename T>
struct OpAxmy {
  using Arg = VecArg<T>;
  static __device__ void apply(const Arg& a, int t, int j) {
    const T c = (T)a.s[j];
    a.x[t] = a.y[t] - c * a.z[t];
  }
};

// x = x + alpha y + omega z
template <typename T>
struct OpBicgX {
  using Arg = VecArg<T>;
  static __device__ void apply(const Arg& a, int t, int) {
    const T alpha = (T)a.s[2], omega = (T)a.s[3];
    a.x[t] = a.x[t] + alpha * a.y[t] + omega * a.z[t];
  }
};

struct MixArg {
  double* d;
  float* f;
};

struct OpToF32 {
  using Arg = MixArg;
  static __device__ void apply(const Arg& a, int t, int) { a.f[t] = (float)a.d[t]; }
};

// the defect-correction update x += e
struct OpAddF32 {
  using Arg = MixArg;
  static __device__ void apply(const Arg& a, int t, int) { a.d[t] += (double)a.f[t]; }
};

// x -= (mean), the mean being *s scaled by inv
struct MeanArg {
  double* x;
  const double* s;
  double inv;
};

struct OpSubMean {
  using Arg = MeanArg;
  static __device__ void apply(const Arg& a, int t, int) {
    const double m = *a.s * a.inv;
    a.x[t] -= m;
  }
};

// ---------------------------------------------------------------------------
// exact coarsest-level solves, one block per cavity
// ---------------------------------------------------------------------------
// the bottom solves of the cavities whose coarsest level is below `below`
// (the others are solved inside the fused tail of the V-cycle)
template <int D, typename T>
__global__ void __launch_bounds__(128) k_batch_bottom(const BottomArg<T>* __restrict__ args, int ncav,
                                                      const int* __restrict__ mask, int below) {
  const int c = blockIdx.x;
  if (c >= ncav || (mask && !mask[c])) return;
  const BottomArg<T>& a = args[c];
  if (a.level >= below) return;
  bottom_block<D, T>(a);
}

// dense bottom operator of the viscous problem (it changes with eta and dt
// every step) and its inverse, for every cavity in one launch each
struct DenseArg {
  double *X, *M, *A, *Minv;
  int n, m;
  const double* ef[3];
  Geom g;
  double beta;
};

template <int D>
__global__ void k_batch_dense_build(const DenseArg* __restrict__ args, int ncav) {
  const int c = blockIdx.y;
  if (c >= ncav) return;
  const DenseArg& a = args[c];
  if ((int)blockIdx.x >= a.n) return;
  dense_build_col<D>(0, a.X, a.M, a.n, a.m, a.ef[0], a.ef[1], a.ef[2], a.g, a.beta, blockIdx.x);
}

__global__ void k_batch_gauss_jordan(const DenseArg* __restrict__ args, int ncav) {
  const int c = blockIdx.x;
  if (c >= ncav) return;
  const DenseArg& a = args[c];
  gauss_jordan_block(a.M, a.m, a.A, a.Minv);
}

}  // namespace batch
}  // namespace hb

namespace hb {
namespace batch {

// ---------------------------------------------------------------------------
// host helpers: lists, tables, reductions, graphs
// ---------------------------------------------------------------------------
static int bfail(hbf_batch* B, int code, const std::string& m) {
  B->err = m;
  return code;
}

static int bcheck(hbf_batch* B, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HBF_OK;
  return bfail(B, e == cudaErrorMemoryAllocation ? HBF_ERR_OOM : HBF_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

// tiles of `tile` elements over count[c] elements of every cavity c
static int make_list(hbf_batch* B, const std::vector<long long>& count, List& L) {
  std::vector<Tile> h;
  L.first.assign(B->ncav + 1, 0);
  for (int c = 0; c < B->ncav; ++c) {
    L.first[c] = (int)h.size();
    for (long long b = 0; b < count[c]; b += B->tile)
      h.push_back(Tile{c, (int)b, (int)std::min<long long>(b + B->tile, count[c])});
  }
  L.first[B->ncav] = (int)h.size();
  L.n = (int)h.size();
  if (L.n > B->max_tiles) B->max_tiles = L.n;
  void *d = nullptr, *df = nullptr;
  if (L.n > 0) {
    if (cudaMalloc(&d, sizeof(Tile) * h.size()) != cudaSuccess) return bfail(B, HBF_ERR_OOM, "tile list");
    B->lallocs.push_back(d);
    cudaMemcpy(d, h.data(), sizeof(Tile) * h.size(), cudaMemcpyHostToDevice);
  }
  if (cudaMalloc(&df, sizeof(int) * L.first.size()) != cudaSuccess) return bfail(B, HBF_ERR_OOM, "tile list");
  B->lallocs.push_back(df);
  cudaMemcpy(df, L.first.data(), sizeof(int) * L.first.size(), cudaMemcpyHostToDevice);
  L.d = (Tile*)d;
  L.dfirst = (int*)df;
  return HBF_OK;
}

template <int D>
static long long space_count(const Geom& g, int s) {
  switch (s) {
    case kCells: return g.ncell;
    case kCellsD: return (long long)D * g.ncell;
    case kRb: return rb_count<D>(g);
    case kNodes: return g.nnode;
    case kFaces: return (long long)g.nface[0] + g.nface[1] + (D == 3 ? g.nface[2] : 0);
    default: {
      const int col = s - kMc0;
      return col < (1 << D) ? mc_count<D>(g, col) : 0;
    }
  }
}

template <int D>
static int build_lists(hbf_batch* B) {
  B->max_tiles = 0;
  for (int l = 0; l < kMaxLev; ++l)
    for (int s = 0; s < kSpaces; ++s) {
      B->H[l][s] = List();
      B->A[l][s] = List();
    }
  for (int l = 0; l < B->maxlev; ++l)
    for (int s = 0; s < kSpaces; ++s) {
      std::vector<long long> h(B->ncav, 0), a(B->ncav, 0);
      for (int c = 0; c < B->ncav; ++c) {
        if (l < B->nlev[c]) h[c] = space_count<D>(B->cav[c]->lv[l].g, s);
        if (l < B->nlev[c] - 1) a[c] = h[c];
      }
      int st = make_list(B, h, B->H[l][s]);
      if (!st) st = make_list(B, a, B->A[l][s]);
      if (st) return st;
    }
  return HBF_OK;
}

template <class ArgT, class F>
static void* make_table(hbf_batch* B, F f) {
  std::vector<ArgT> h(B->ncav);
  for (int c = 0; c < B->ncav; ++c) h[c] = f(B->cav[c], c);
  return upload_table(B, h);
}

// per-cavity reduction of list L (level 0) into red slot `slot`
template <typename T>
static void reduce(hbf_batch* B, const void* tab, const List& L, int mode, int slot, const int* mask,
                   const double* scale = nullptr) {
  const int wpb = kThreads / 32;  // warps (tiles in flight) per block
  int grid = 152 * B->blocks_per_sm;
  if (grid > (L.n + wpb - 1) / wpb) grid = (L.n + wpb - 1) / wpb;
  if (grid < 1) grid = 1;
  k_batch_reduce<T><<<grid, kThreads, 0, B->stream>>>((const RedArg<T>*)tab, L.d, L.n, mask, mode, B->part);
  k_batch_combine<<<(B->ncav + wpb - 1) / wpb, kThreads, 0, B->stream>>>(B->part, L.dfirst, B->ncav, mode, scale,
                                                                         B->red + (size_t)slot * B->ncav);
  B->nlaunch += 2;
}

// bring the first nslots result slots to the host
static int fetch(hbf_batch* B, int nslots) {
  cudaError_t e = cudaMemcpyAsync(B->hred, B->red, sizeof(double) * nslots * B->ncav, cudaMemcpyDeviceToHost,
                                  B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  B->h2d_pending = false;
  return bcheck(B, e, "batched reduction");
}

static double hr(hbf_batch* B, int slot, int c) { return B->hred[(size_t)slot * B->ncav + c]; }

// active-cavity mask: uploaded only when it changed (always after a
// synchronisation, so the pinned buffer is free to rewrite)
static void h2d_wait(hbf_batch* B) {
  if (B->h2d_pending) cudaStreamSynchronize(B->stream);
  B->h2d_pending = false;
}

static void set_mask(hbf_batch* B, const std::vector<char>& on) {
  bool same = (int)B->act_uploaded.size() == B->ncav;
  for (int c = 0; c < B->ncav && same; ++c) same = B->act_uploaded[c] == (on[c] ? 1 : 0);
  if (same) return;
  h2d_wait(B);
  B->act_uploaded.assign(B->ncav, 0);
  for (int c = 0; c < B->ncav; ++c) B->h_act[c] = B->act_uploaded[c] = on[c] ? 1 : 0;
  cudaMemcpyAsync(B->mask_act, B->h_act, sizeof(int) * B->ncav, cudaMemcpyHostToDevice, B->stream);
  B->h2d_pending = true;
}

// the host writes hscal only after a fetch (or h2d_wait) since the last upload
static void upload_scalars(hbf_batch* B) {
  cudaMemcpyAsync(B->scal, B->hscal, sizeof(double) * 4 * B->ncav, cudaMemcpyHostToDevice, B->stream);
  B->h2d_pending = true;
}

static bool any(const std::vector<char>& v) {
  for (char x : v)
    if (x) return true;
  return false;
}

// a fixed launch sequence, captured once and replayed
struct Graph {
  cudaGraphExec_t exec = nullptr;
  long long nk = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    nk = 0;
  }
};

template <class F>
static int replay(hbf_batch* B, Graph& G, F body) {
  if (!G.exec) {
    const long long n0 = B->nlaunch;
    cudaError_t e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcheck(B, e, "graph capture");
    body();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->stream, &g);
    if (e != cudaSuccess) return bcheck(B, e, "graph capture");
    e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      G.exec = nullptr;
      return bcheck(B, e, "graph instantiate");
    }
    G.nk = B->nlaunch - n0;
    B->nlaunch = n0;
  }
  B->nlaunch += G.nk;
  return bcheck(B, cudaGraphLaunch(G.exec, B->stream), "graph launch");
}

// per-precision level arrays
template <typename T>
struct LvView;
template <>
struct LvView<double> {
  static double* vx(Level& L) { return L.vx; }
  static double* vb(Level& L) { return L.vb; }
  static double* vr(Level& L) { return L.vr; }
  static const double* ef(Level& L, int a) { return L.ef[a]; }
  static double* cx(Level& L) { return L.cx; }
  static double* cb(Level& L) { return L.cb; }
  static double* cr(Level& L) { return L.cr; }
  static double* nx(Level& L) { return L.nx; }
  static double* nb(Level& L) { return L.nb; }
  static double* nr(Level& L) { return L.nr; }
};
template <>
struct LvView<float> {
  static float* vx(Level& L) { return L.fvx; }
  static float* vb(Level& L) { return L.fvb; }
  static float* vr(Level& L) { return L.fvr; }
  static const float* ef(Level& L, int a) { return L.fef[a]; }
  static float* cx(Level& L) { return L.fcx; }
  static float* cb(Level& L) { return L.fcb; }
  static float* cr(Level& L) { return L.fcr; }
  static float* nx(Level& L) { return L.fnx; }
  static float* nb(Level& L) { return L.fnb; }
  static float* nr(Level& L) { return L.fnr; }
};

// ---------------------------------------------------------------------------
// one linear problem on every cavity's hierarchy: the argument tables of its
// V-cycle (level 0 iterate and right-hand side given per cavity)
// ---------------------------------------------------------------------------

struct Inst {
  int kind = 0;
  TailTabs tail = {};
  void* lv[kMaxLev] = {};  // smoother / residual arguments of level l
  void* re[kMaxLev] = {};  // restriction l -> l+1
  void* pr[kMaxLev] = {};  // prolongation l+1 -> l
  void* bot = nullptr;     // bottom solve
  Graph g;
};

template <int D, typename T>
static void build_inst(hbf_batch* B, Inst& I, int kind, bool hom0, T* (*x0)(hbf_ctx*), T* (*b0)(hbf_ctx*)) {
  using V = LvView<T>;
  I.kind = kind;
  auto X = [&](hbf_ctx* c, int l) -> T* {
    Level& L = c->lv[l];
    if (l == 0) return x0(c);
    return kind == kVisc ? V::vx(L) : kind == kMac ? V::cx(L) : V::nx(L);
  };
  auto Bv = [&](hbf_ctx* c, int l) -> T* {
    Level& L = c->lv[l];
    if (l == 0) return b0(c);
    return kind == kVisc ? V::vb(L) : kind == kMac ? V::cb(L) : V::nb(L);
  };
  auto R = [&](hbf_ctx* c, int l) -> T* {
    Level& L = c->lv[l];
    return kind == kVisc ? V::vr(L) : kind == kMac ? V::cr(L) : V::nr(L);
  };
  for (int l = 0; l < B->maxlev; ++l) {
    if (kind == kVisc)
      I.lv[l] = make_table<ViscArg<T>>(B, [&](hbf_ctx* c, int q) {
        ViscArg<T> a;
        std::memset(&a, 0, sizeof a);
        if (l >= B->nlev[q]) return a;
        Level& L = c->lv[l];
        a.x = X(c, l);
        a.b = Bv(c, l);
        a.out = R(c, l);
        for (int d = 0; d < 3; ++d) a.ef[d] = d < D ? V::ef(L, d) : nullptr;
        a.g = L.g;
        a.beta = (T)visc_beta(B->dt[q], c->rho, c->theta);
        a.hom = (l > 0 || hom0) ? 1 : 0;
        return a;
      });
    else
      I.lv[l] = make_table<PoisArg<T>>(B, [&](hbf_ctx* c, int q) {
        PoisArg<T> a;
        std::memset(&a, 0, sizeof a);
        if (l >= B->nlev[q]) return a;
        a.x = X(c, l);
        a.b = Bv(c, l);
        a.r = R(c, l);
        a.g = c->lv[l].g;
        return a;
      });
    if (l + 1 < B->maxlev) {
      I.re[l] = make_table<XferArg<T>>(B, [&](hbf_ctx* c, int q) {
        XferArg<T> a;
        std::memset(&a, 0, sizeof a);
        if (l + 1 >= B->nlev[q]) return a;
        a.src = R(c, l);
        a.dst = Bv(c, l + 1);
        a.zero = X(c, l + 1);
        a.gf = c->lv[l].g;
        a.gc = c->lv[l + 1].g;
        a.ncomp = kind == kVisc ? D : 1;
        a.sign = kind == kVisc ? -1 : 1;
        return a;
      });
      I.pr[l] = make_table<XferArg<T>>(B, [&](hbf_ctx* c, int q) {
        XferArg<T> a;
        std::memset(&a, 0, sizeof a);
        if (l + 1 >= B->nlev[q]) return a;
        a.src = X(c, l + 1);
        a.dst = X(c, l);
        a.gf = c->lv[l].g;
        a.gc = c->lv[l + 1].g;
        a.ncomp = kind == kVisc ? D : 1;
        a.sign = kind == kVisc ? -1 : 1;
        return a;
      });
    }
  }
  I.bot = make_table<BottomArg<T>>(B, [&](hbf_ctx* c, int q) {
    const int l = B->nlev[q] - 1;
    const Geom& g = c->lv[l].g;
    BottomArg<T> a;
    a.n = kind == kVisc ? D * g.ncell : kind == kMac ? g.ncell : g.nnode;
    a.m = kind == kVisc ? a.n : a.n + 1;
    a.Minv = c->dense[kind].Minv;
    a.x = X(c, l);
    a.b = Bv(c, l);
    a.g = g;
    a.kind = kind;
    a.level = l;
    return a;
  });
  for (int l = 0; l < kMaxLev; ++l) {
    I.tail.lv[l] = I.lv[l];
    I.tail.re[l] = I.re[l];
    I.tail.pr[l] = I.pr[l];
  }
  I.tail.bot = I.bot;
}

template <int D, typename T>
static void smooth(hbf_batch* B, Inst& I, int l, const int* mask) {
  if (I.kind == kVisc) {
    for (int col = 0; col < 2; ++col) run<OpViscSmooth<D, T, 0>>(B, I.lv[l], B->A[l][kRb], mask, col);
    for (int col = 0; col < 2; ++col) run<OpViscSmooth<D, T, 1>>(B, I.lv[l], B->A[l][kRb], mask, col);
    if (D == 3)
      for (int col = 0; col < 2; ++col) run<OpViscSmooth<D, T, (D == 3 ? 2 : 0)>>(B, I.lv[l], B->A[l][kRb], mask, col);
  } else if (I.kind == kMac) {
    for (int col = 0; col < 2; ++col) run<OpCellSmooth<D, T>>(B, I.lv[l], B->A[l][kRb], mask, col);
  } else {
    for (int col = 0; col < (1 << D); ++col) run<OpNodalSmooth<D, T>>(B, I.lv[l], B->A[l][kMc0 + col], mask, col);
  }
}

// V(nu1, nu2) cycle of every masked cavity at once: descend through the
// levels that are not a cavity's coarsest, one batched exact bottom solve,
// ascend
template <int D, typename T>
static void vcycle(hbf_batch* B, Inst& I, const int* mask) {
  const SolverCfg& cfg = B->cav[0]->cfg;
  const int lf = B->tail_level;  // levels >= lf run in the fused tail kernel
  int top = 0;  // levels 0 .. top-1 descend level by level
  while (top < B->maxlev - 1 && top < lf && B->A[top][kCells].n > 0) ++top;
  for (int l = 0; l < top; ++l) {
    for (int s = 0; s < cfg.nu1; ++s) smooth<D, T>(B, I, l, mask);
    if (I.kind == kVisc) {
      run<OpViscOp<D, T>>(B, I.lv[l], B->A[l][kCells], mask);
      run<OpRestrictCells<D, T>>(B, I.re[l], B->H[l + 1][kCellsD], mask);
    } else if (I.kind == kMac) {
      run<OpCellResid<D, T>>(B, I.lv[l], B->A[l][kCells], mask);
      run<OpRestrictCells<D, T>>(B, I.re[l], B->H[l + 1][kCells], mask);
    } else {
      run<OpNodalResid<D, T>>(B, I.lv[l], B->A[l][kNodes], mask);
      run<OpRestrictNodes<D, T>>(B, I.re[l], B->H[l + 1][kNodes], mask);
    }
  }
  k_batch_bottom<D, T><<<B->ncav, 128, 0, B->stream>>>((const BottomArg<T>*)I.bot, B->ncav, mask, lf);
  ++B->nlaunch;
  if (lf < B->maxlev) {
    if (I.kind == kVisc)
      k_vcycle_tail<D, T, kVisc, false><<<B->ncav, 256, 0, B->stream>>>(I.tail, lf, B->ncav, mask, cfg.nu1, cfg.nu2);
    else if (I.kind == kMac)
      k_vcycle_tail<D, T, kMac, false><<<B->ncav, 256, 0, B->stream>>>(I.tail, lf, B->ncav, mask, cfg.nu1, cfg.nu2);
    else
      k_vcycle_tail<D, T, kNodal, false><<<B->ncav, 256, 0, B->stream>>>(I.tail, lf, B->ncav, mask, cfg.nu1,
                                                                         cfg.nu2);
    ++B->nlaunch;
  }
  for (int l = top - 1; l >= 0; --l) {
    if (I.kind == kVisc)
      run<OpProlongCells<D, T>>(B, I.pr[l], B->A[l][kCellsD], mask);
    else if (I.kind == kMac)
      run<OpProlongCells<D, T>>(B, I.pr[l], B->A[l][kCells], mask);
    else
      run<OpProlongNodes<D, T>>(B, I.pr[l], B->A[l][kNodes], mask);
    for (int s = 0; s < cfg.nu2; ++s) smooth<D, T>(B, I, l, mask);
  }
}

}  // namespace batch
}  // namespace hb

namespace hb {
namespace batch {

// ---------------------------------------------------------------------------
// the step of every cavity: argument tables and the host loops
// ---------------------------------------------------------------------------
constexpr double kInnerRtol = 1e-3;  // mixed viscous solve: inner residual drop
constexpr int kInnerMax = 40;        // and inner iteration cap (as the single-cavity solve)

// Krylov vectors of the viscous solve in the solver arithmetic T
template <typename T>
struct KV;
template <>
struct KV<double> {
  static double* r(hbf_ctx* c) { return c->kr; }
  static double* rh(hbf_ctx* c) { return c->krh; }
  static double* p(hbf_ctx* c) { return c->kp; }
  static double* v(hbf_ctx* c) { return c->kv; }
  static double* s(hbf_ctx* c) { return c->ks; }
  static double* t(hbf_ctx* c) { return c->kt; }
  static double* ph(hbf_ctx* c) { return c->kph; }
  static double* sh(hbf_ctx* c) { return c->ksh; }
  static double* x(hbf_ctx* c) { return c->ustar; }
  static double* macx(hbf_ctx* c) { return c->phi_mac; }
  static double* macb(hbf_ctx* c) { return c->lv[0].cb; }
  static double* nodx(hbf_ctx* c) { return c->p; }
  static double* nodb(hbf_ctx* c) { return c->lv[0].nb; }
};
template <>
struct KV<float> {
  static float* r(hbf_ctx* c) { return c->fkr; }
  static float* rh(hbf_ctx* c) { return c->fkrh; }
  static float* p(hbf_ctx* c) { return c->fkp; }
  static float* v(hbf_ctx* c) { return c->fkv; }
  static float* s(hbf_ctx* c) { return c->fks; }
  static float* t(hbf_ctx* c) { return c->fkt; }
  static float* ph(hbf_ctx* c) { return c->fkph; }
  static float* sh(hbf_ctx* c) { return c->fksh; }
  static float* x(hbf_ctx* c) { return c->fke; }
  static float* macx(hbf_ctx* c) { return c->lv[0].fcx; }
  static float* macb(hbf_ctx* c) { return c->lv[0].fcb; }
  static float* nodx(hbf_ctx* c) { return c->lv[0].fnx; }
  static float* nodb(hbf_ctx* c) { return c->lv[0].fnb; }
};

struct Solvers {
  virtual ~Solvers() {}
  virtual int step(hbf_batch* B, hbf_step_stats* st) = 0;
  // a representative launch sequence that changes no cavity state (tuning)
  virtual int probe(hbf_batch* B) = 0;
};

template <typename T>
static VecArg<T> vec(T* x, const T* y = nullptr, const T* z = nullptr, const double* s = nullptr) {
  return VecArg<T>{x, y, z, s};
}

template <int D, typename T>
struct SolversT : Solvers {
  static constexpr bool kMixed = sizeof(T) == 4;
  using K = KV<T>;
  Inst vph, vsh, mac, nod;
  // explicit stages and the viscous preparation
  void *tlu = nullptr, *zero_phi = nullptr, *dense = nullptr, *cp_in = nullptr, *cp_out = nullptr;
  void* facesR[kMaxLev] = {};
  void* facesF[kMaxLev] = {};
  // MAC (0) and nodal (1) solves, level-0 tables
  struct MG {
    void *copyb, *sumb, *subb, *sumx, *subx, *redb, *res64, *redr, *tof, *zerof, *add;
  } mg[2];
  // viscous solve
  void *v_copyb, *v_redb, *v_true, *v_redr;
  void *k_tof, *k_zero_x, *k_copy_rh, *k_zero_v, *k_zero_p, *k_red_r0, *k_dot_rh_r, *k_bicg_p, *k_zero_ph,
      *k_apply_ph, *k_dot_rh_v, *k_axmy_s, *k_zero_sh, *k_apply_sh, *k_dot_tt, *k_dot_ts, *k_bicg_x, *k_axmy_r,
      *k_red_r, *k_add;
  Graph g_pre, g_post, g_nrhs, g_upd;

  ~SolversT() override {
    for (Graph* g : {&g_pre, &g_post, &g_nrhs, &g_upd, &vph.g, &vsh.g, &mac.g, &nod.g}) g->reset();
  }

  void build(hbf_batch* B) {
    const int n = B->ncav;
    auto S = [B](int c) { return (const double*)(B->scal + 4 * (size_t)c); };
    auto M = [B](int slot, int c) { return (const double*)(B->red + (size_t)slot * B->ncav + c); };
    (void)n;
    // V-cycle problems: viscous preconditioner on p -> ph and s -> sh,
    // MAC and nodal corrections
    build_inst<D, T>(B, vph, kVisc, true, &K::ph, &K::p);
    build_inst<D, T>(B, vsh, kVisc, true, &K::sh, &K::s);
    build_inst<D, T>(B, mac, kMac, true, &K::macx, &K::macb);
    build_inst<D, T>(B, nod, kNodal, true, &K::nodx, &K::nodb);
    // explicit-stage extras
    tlu = make_table<ViscArg<double>>(B, [&](hbf_ctx* c, int) {
      ViscArg<double> a;
      std::memset(&a, 0, sizeof a);
      a.x = c->u;
      a.out = c->Lu;
      for (int d = 0; d < D; ++d) a.ef[d] = c->lv[0].ef[d];
      a.g = c->g;
      return a;
    });
    zero_phi = make_table<VecArg<double>>(B, [&](hbf_ctx* c, int) { return vec<double>(c->phi_mac); });
    cp_in = make_table<VecArg<double>>(B, [&](hbf_ctx* c, int) { return vec<double>(c->ustar, c->u); });
    cp_out = make_table<VecArg<double>>(B, [&](hbf_ctx* c, int) { return vec<double>(c->u, c->ustar); });
    for (int l = 0; l < B->maxlev; ++l) {
      facesF[l] = make_table<FaceArg>(B, [&](hbf_ctx* c, int q) {
        FaceArg a;
        std::memset(&a, 0, sizeof a);
        if (l >= B->nlev[q]) return a;
        for (int d = 0; d < D; ++d) {
          a.src[d] = c->lv[l].ef[d];
          a.fdst[d] = c->lv[l].fef[d];
        }
        a.gf = c->lv[l].g;
        return a;
      });
      if (l + 1 < B->maxlev)
        facesR[l] = make_table<FaceArg>(B, [&](hbf_ctx* c, int q) {
          FaceArg a;
          std::memset(&a, 0, sizeof a);
          if (l + 1 >= B->nlev[q]) return a;
          for (int d = 0; d < D; ++d) {
            a.src[d] = c->lv[l].ef[d];
            a.dst[d] = c->lv[l + 1].ef[d];
          }
          a.gf = c->lv[l].g;
          a.gc = c->lv[l + 1].g;
          return a;
        });
    }
    dense = make_table<DenseArg>(B, [&](hbf_ctx* c, int q) {
      const Level& L = c->lv[B->nlev[q] - 1];
      DenseArg a;
      std::memset(&a, 0, sizeof a);
      a.X = c->dX;
      a.M = c->dM;
      a.A = c->dA;
      a.Minv = c->dense[0].Minv;
      a.n = a.m = D * L.g.ncell;
      for (int d = 0; d < D; ++d) a.ef[d] = L.ef[d];
      a.g = L.g;
      a.beta = visc_beta(B->dt[q], c->rho, c->theta);
      return a;
    });
    // MAC and nodal solves
    for (int w = 0; w < 2; ++w) {
      MG& G = mg[w];
      auto X64 = [w](hbf_ctx* c) { return w == 0 ? c->phi_mac : c->p; };
      auto B64 = [w](hbf_ctx* c) { return w == 0 ? c->lv[0].cb : c->lv[0].nb; };
      auto R64 = [w](hbf_ctx* c) { return w == 0 ? c->lv[0].cr : c->lv[0].nr; };
      auto RHS = [w](hbf_ctx* c) { return w == 0 ? c->mrhs : c->nrhs; };
      auto inv = [w, D_ = D](hbf_ctx* c) {
        return w == 0 ? 1.0 / (double)c->g.ncell
                      : 1.0 / ((double)c->g.n[0] * c->g.n[1] * (D_ == 3 ? c->g.n[2] : 1));
      };
      G.copyb = make_table<VecArg<double>>(B, [&](hbf_ctx* c, int) { return vec<double>(B64(c), RHS(c)); });
      G.sumb = make_table<RedArg<double>>(B, [&](hbf_ctx* c, int) { return RedArg<double>{B64(c), nullptr, c->g, D}; });
      G.sumx = make_table<RedArg<double>>(B, [&](hbf_ctx* c, int) { return RedArg<double>{X64(c), nullptr, c->g, D}; });
      G.subb = make_table<MeanArg>(B, [&](hbf_ctx* c, int q) { return MeanArg{B64(c), M(3, q), inv(c)}; });
      G.subx = make_table<MeanArg>(B, [&](hbf_ctx* c, int q) { return MeanArg{X64(c), M(3, q), inv(c)}; });
      G.redb = G.sumb;
      G.redr = make_table<RedArg<double>>(B, [&](hbf_ctx* c, int) { return RedArg<double>{R64(c), nullptr, c->g, D}; });
      G.res64 = make_table<PoisArg<double>>(B, [&](hbf_ctx* c, int) { return PoisArg<double>{X64(c), B64(c), R64(c), c->g}; });
      G.tof = G.zerof = G.add = nullptr;
      if (kMixed) {
        G.tof = make_table<MixArg>(B, [&](hbf_ctx* c, int) {
          return MixArg{R64(c), w == 0 ? c->lv[0].fcb : c->lv[0].fnb};
        });
        G.zerof = make_table<VecArg<float>>(B, [&](hbf_ctx* c, int) {
          return vec<float>(w == 0 ? c->lv[0].fcx : c->lv[0].fnx);
        });
        G.add = make_table<MixArg>(B, [&](hbf_ctx* c, int) {
          return MixArg{X64(c), w == 0 ? c->lv[0].fcx : c->lv[0].fnx};
        });
      }
    }
    // viscous solve
    v_copyb = make_table<VecArg<double>>(B, [&](hbf_ctx* c, int) { return vec<double>(c->kb, c->rhs); });
    v_redb = make_table<RedArg<double>>(B, [&](hbf_ctx* c, int) { return RedArg<double>{c->kb, nullptr, c->g, D}; });
    v_redr = make_table<RedArg<double>>(B, [&](hbf_ctx* c, int) { return RedArg<double>{c->kr, nullptr, c->g, D}; });
    v_true = make_table<ViscArg<double>>(B, [&](hbf_ctx* c, int q) {
      ViscArg<double> a;
      std::memset(&a, 0, sizeof a);
      a.x = c->ustar;
      a.b = c->kb;
      a.out = c->kr;
      for (int d = 0; d < D; ++d) a.ef[d] = c->lv[0].ef[d];
      a.g = c->g;
      a.beta = visc_beta(B->dt[q], c->rho, c->theta);
      a.hom = 0;
      return a;
    });
    auto apply = [&](T* (*in)(hbf_ctx*), T* (*outp)(hbf_ctx*)) {
      return make_table<ViscArg<T>>(B, [&](hbf_ctx* c, int q) {
        ViscArg<T> a;
        std::memset(&a, 0, sizeof a);
        a.x = in(c);
        a.b = nullptr;
        a.out = outp(c);
        for (int d = 0; d < D; ++d) a.ef[d] = LvView<T>::ef(c->lv[0], d);
        a.g = c->g;
        a.beta = (T)visc_beta(B->dt[q], c->rho, c->theta);
        a.hom = 1;
        return a;
      });
    };
    auto red = [&](T* (*x)(hbf_ctx*), T* (*y)(hbf_ctx*)) {
      return make_table<RedArg<T>>(B, [&](hbf_ctx* c, int) { return RedArg<T>{x(c), y ? y(c) : nullptr, c->g, D}; });
    };
    auto vt = [&](T* (*x)(hbf_ctx*), T* (*y)(hbf_ctx*), T* (*z)(hbf_ctx*)) {
      return make_table<VecArg<T>>(B, [&](hbf_ctx* c, int q) {
        return vec<T>(x(c), y ? y(c) : nullptr, z ? z(c) : nullptr, S(q));
      });
    };
    k_tof = kMixed ? make_table<MixArg>(B, [&](hbf_ctx* c, int) { return MixArg{c->kr, c->fkr}; }) : nullptr;
    k_add = kMixed ? make_table<MixArg>(B, [&](hbf_ctx* c, int) { return MixArg{c->ustar, c->fke}; }) : nullptr;
    k_zero_x = vt(&K::x, nullptr, nullptr);
    k_copy_rh = vt(&K::rh, &K::r, nullptr);
    k_zero_v = vt(&K::v, nullptr, nullptr);
    k_zero_p = vt(&K::p, nullptr, nullptr);
    k_red_r0 = red(&K::r, nullptr);
    k_dot_rh_r = red(&K::rh, &K::r);
    k_bicg_p = vt(&K::p, &K::r, &K::v);
    k_zero_ph = vt(&K::ph, nullptr, nullptr);
    k_apply_ph = apply(&K::ph, &K::v);
    k_dot_rh_v = red(&K::rh, &K::v);
    k_axmy_s = vt(&K::s, &K::r, &K::v);
    k_zero_sh = vt(&K::sh, nullptr, nullptr);
    k_apply_sh = apply(&K::sh, &K::t);
    k_dot_tt = red(&K::t, &K::t);
    k_dot_ts = red(&K::t, &K::s);
    k_bicg_x = vt(&K::x, &K::ph, &K::sh);
    k_axmy_r = vt(&K::r, &K::s, &K::t);
    k_red_r = k_red_r0;
  }

  int vcyc(hbf_batch* B, Inst& I) {
    return replay(B, I.g, [&] { vcycle<D, T>(B, I, B->mask_act); });
  }

  // coarse face viscosity of every level, FP32 copies, and the exact inverse
  // of each cavity's viscous bottom operator
  void prep_visc(hbf_batch* B) {
    for (int l = 0; l + 1 < B->maxlev; ++l)
      run<OpRestrictFaces<D>>(B, facesR[l], B->H[l + 1][kFaces], B->mask_all);
    if (kMixed)
      for (int l = 0; l < B->maxlev; ++l) run<OpFacesF32>(B, facesF[l], B->H[l][kFaces], B->mask_all);
    k_batch_dense_build<D><<<dim3(kDenseMax, B->ncav), 128, 0, B->stream>>>((const DenseArg*)dense, B->ncav);
    k_batch_gauss_jordan<<<B->ncav, 256, 0, B->stream>>>((const DenseArg*)dense, B->ncav);
    B->nlaunch += 2;
  }

  // MAC (w = 0) or nodal (w = 1) projection solve: multigrid, or FP64 defect
  // correction around FP32 V-cycles, per cavity to its own tolerance
  int mg_solve(hbf_batch* B, int w, hbf_solve_stats* out) {
    MG& G = mg[w];
    Inst& I = w == 0 ? mac : nod;
    const List& L0 = w == 0 ? B->H[0][kCells] : B->H[0][kNodes];
    const int msum = w == 0 ? 1 : 3;
    const int* all = B->mask_all;
    const int* act_d = B->mask_act;
    auto resid = [&](const int* m) {
      if (w == 0)
        run<OpCellResid<D, double>>(B, G.res64, L0, m);
      else
        run<OpNodalResid<D, double>>(B, G.res64, L0, m);
    };
    run<OpCopy<double>>(B, G.copyb, L0, all);
    reduce<double>(B, G.sumb, L0, msum, 3, all);
    run<OpSubMean>(B, G.subb, L0, all);
    reduce<double>(B, G.sumx, L0, msum, 3, all);
    run<OpSubMean>(B, G.subx, L0, all);
    reduce<double>(B, G.redb, L0, 0, 0, all);
    resid(all);
    reduce<double>(B, G.redr, L0, 0, 1, all);
    int st = fetch(B, 2);
    if (st) return st;
    const int n = B->ncav;
    std::vector<double> bnorm(n), rn(n), r0(n), tol(n);
    std::vector<int> cyc(n, 0);
    std::vector<char> act(n, 0);
    for (int c = 0; c < n; ++c) {
      bnorm[c] = hr(B, 0, c);
      rn[c] = r0[c] = hr(B, 1, c);
      if (bnorm[c] == 0.0) bnorm[c] = rn[c];
      tol[c] = B->cav[c]->cfg.rtol * bnorm[c];
      act[c] = rn[c] > tol[c] && cyc[c] < B->cav[c]->cfg.max_cycles && std::isfinite(rn[c]);
    }
    while (any(act)) {
      ++B->trips[w == 0 ? 0 : 2];
      set_mask(B, act);
      if (kMixed) {
        run<OpToF32>(B, G.tof, L0, act_d);
        run<OpZero<float>>(B, G.zerof, L0, act_d);
        if ((st = vcyc(B, I))) return st;
        run<OpAddF32>(B, G.add, L0, act_d);
      } else {
        if ((st = vcyc(B, I))) return st;
      }
      reduce<double>(B, G.sumx, L0, msum, 3, act_d);
      run<OpSubMean>(B, G.subx, L0, act_d);
      resid(act_d);
      reduce<double>(B, G.redr, L0, 0, 1, act_d);
      if ((st = fetch(B, 2))) return st;
      for (int c = 0; c < n; ++c)
        if (act[c]) {
          ++cyc[c];
          rn[c] = hr(B, 1, c);
          act[c] = rn[c] > tol[c] && cyc[c] < B->cav[c]->cfg.max_cycles && std::isfinite(rn[c]);
        }
    }
    return finish(B, out, w == 0 ? "MAC" : "nodal", cyc, r0, rn, bnorm, tol);
  }

  static int finish(hbf_batch* B, hbf_solve_stats* out, const char* what, const std::vector<int>& it,
                    const std::vector<double>& r0, const std::vector<double>& rn, const std::vector<double>& bnorm,
                    const std::vector<double>& tol) {
    int worst = HBF_OK;
    for (int c = 0; c < B->ncav; ++c) {
      hbf_solve_stats s;
      s.cycles = it[c];
      s.r0 = r0[c];
      s.rnorm = rn[c];
      s.bnorm = bnorm[c];
      s.converged = rn[c] <= tol[c];
      s.guess = 0;
      if (out) out[c] = s;
      char buf[160];
      if (!std::isfinite(rn[c]) || !std::isfinite(bnorm[c])) {
        snprintf(buf, sizeof buf, "%s solve of cavity %d: non-finite residual norm", what, c);
        B->err = buf;
        return HBF_ERR_NONFINITE;
      }
      if (!s.converged && worst == HBF_OK) {
        snprintf(buf, sizeof buf, "%s solve of cavity %d did not converge: %d cycles, residual %.3e > tol %.3e",
                 what, c, it[c], rn[c], tol[c]);
        B->err = buf;
        worst = HBF_ERR_NOT_CONVERGED;
      }
    }
    return worst;
  }

  // (I - beta L_eta) u = rhs by BiCGStab right-preconditioned with one
  // homogeneous V-cycle; in mixed arithmetic FP64 defect correction around an
  // FP32 BiCGStab.  Same per-cavity iteration as the single-cavity solve.
  int visc_solve(hbf_batch* B, hbf_solve_stats* out) {
    const List& Lv = B->H[0][kCellsD];
    const List& Lc = B->H[0][kCells];
    const int* all = B->mask_all;
    const int* act_d = B->mask_act;
    const int n = B->ncav;
    run<OpCopy<double>>(B, v_copyb, Lv, all);
    reduce<double>(B, v_redb, Lv, 0, 0, all);
    run<OpViscOp<D, double>>(B, v_true, Lc, all);
    reduce<double>(B, v_redr, Lv, 0, 1, all);
    int st = fetch(B, 2);
    if (st) return st;
    std::vector<double> bnorm(n), rn(n), r0(n), tol(n), itol(n), rho(n), alpha(n), omega(n), rho1(n), rho1n(n);
    std::vector<int> it(n, 0), k(n, 0);
    std::vector<char> outer(n, 0), inner(n, 0);
    auto cap = [&](int c) { return B->cav[c]->cfg.max_cycles; };
    for (int c = 0; c < n; ++c) {
      bnorm[c] = hr(B, 0, c);
      rn[c] = r0[c] = hr(B, 1, c);
      if (bnorm[c] == 0.0) bnorm[c] = rn[c];
      tol[c] = B->cav[c]->cfg.rtol * bnorm[c];
      outer[c] = rn[c] > tol[c] && it[c] < cap(c) && std::isfinite(rn[c]);
    }
    while (any(outer)) {
      set_mask(B, outer);
      if (kMixed) {
        run<OpToF32>(B, k_tof, Lv, act_d);
        run<OpZero<T>>(B, k_zero_x, Lv, act_d);
        run<OpCopy<T>>(B, k_copy_rh, Lv, act_d);
        run<OpZero<T>>(B, k_zero_v, Lv, act_d);
        run<OpZero<T>>(B, k_zero_p, Lv, act_d);
        reduce<T>(B, k_red_r0, Lv, 0, 0, act_d);
      } else {
        run<OpCopy<T>>(B, k_copy_rh, Lv, act_d);
        run<OpZero<T>>(B, k_zero_v, Lv, act_d);
        run<OpZero<T>>(B, k_zero_p, Lv, act_d);
      }
      // rho1 = (rh, r) of the first inner iteration (outer cavities are exactly
      // the ones entering it); later ones arrive with the residual norm of the
      // previous iteration (same r, one fetch)
      reduce<T>(B, k_dot_rh_r, Lv, 2, 1, act_d);
      if ((st = fetch(B, 2))) return st;
      for (int c = 0; c < n; ++c) {
        if (!outer[c]) {
          inner[c] = 0;
          continue;
        }
        itol[c] = kMixed ? kInnerRtol * hr(B, 0, c) : tol[c];
        rho[c] = alpha[c] = omega[c] = 1.0;
        k[c] = 0;
        inner[c] = it[c] < cap(c);
        rho1n[c] = hr(B, 1, c);
      }
      while (any(inner)) {
        ++B->trips[1];
        for (int c = 0; c < n; ++c)
          if (inner[c]) {
            rho1[c] = rho1n[c];
            if (rho1[c] == 0.0 || !std::isfinite(rho1[c])) {
              inner[c] = 0;
              continue;
            }
            B->hscal[4 * c + 0] = (rho1[c] / rho[c]) * (alpha[c] / omega[c]);
            B->hscal[4 * c + 1] = omega[c];
          }
        if (!any(inner)) break;
        set_mask(B, inner);
        upload_scalars(B);
        run<OpBicgP<T>>(B, k_bicg_p, Lv, act_d);
        run<OpZero<T>>(B, k_zero_ph, Lv, act_d);
        if ((st = vcyc(B, vph))) return st;
        run<OpViscOp<D, T>>(B, k_apply_ph, Lc, act_d);
        reduce<T>(B, k_dot_rh_v, Lv, 2, 0, act_d);
        if ((st = fetch(B, 1))) return st;
        for (int c = 0; c < n; ++c)
          if (inner[c]) {
            const double den = hr(B, 0, c);
            if (den == 0.0 || !std::isfinite(den)) {
              inner[c] = 0;
              continue;
            }
            alpha[c] = rho1[c] / den;
            B->hscal[4 * c + 2] = alpha[c];
          }
        if (!any(inner)) break;
        set_mask(B, inner);
        upload_scalars(B);
        run<OpAxmy<T>>(B, k_axmy_s, Lv, act_d, 2);
        run<OpZero<T>>(B, k_zero_sh, Lv, act_d);
        if ((st = vcyc(B, vsh))) return st;
        run<OpViscOp<D, T>>(B, k_apply_sh, Lc, act_d);
        reduce<T>(B, k_dot_tt, Lv, 2, 0, act_d);
        reduce<T>(B, k_dot_ts, Lv, 2, 1, act_d);
        if ((st = fetch(B, 2))) return st;
        for (int c = 0; c < n; ++c)
          if (inner[c]) {
            const double tt = hr(B, 0, c), ts = hr(B, 1, c);
            omega[c] = tt > 0.0 ? ts / tt : 0.0;
            B->hscal[4 * c + 3] = omega[c];
          }
        upload_scalars(B);
        run<OpBicgX<T>>(B, k_bicg_x, Lv, act_d);
        run<OpAxmy<T>>(B, k_axmy_r, Lv, act_d, 3);
        reduce<T>(B, k_red_r, Lv, 0, 0, act_d);
        reduce<T>(B, k_dot_rh_r, Lv, 2, 1, act_d);
        if ((st = fetch(B, 2))) return st;
        for (int c = 0; c < n; ++c)
          if (inner[c]) {
            rho[c] = rho1[c];
            ++it[c];
            ++k[c];
            const double rr = hr(B, 0, c);
            rho1n[c] = hr(B, 1, c);
            const bool stop = rr <= itol[c] || omega[c] == 0.0 || !std::isfinite(rr);
            inner[c] = !stop && it[c] < cap(c) && (!kMixed || k[c] < kInnerMax);
          }
      }
      set_mask(B, outer);
      if (kMixed) run<OpAddF32>(B, k_add, Lv, act_d);
      run<OpViscOp<D, double>>(B, v_true, Lc, act_d);
      reduce<double>(B, v_redr, Lv, 0, 1, act_d);
      if ((st = fetch(B, 2))) return st;
      for (int c = 0; c < n; ++c)
        if (outer[c]) {
          rn[c] = hr(B, 1, c);
          outer[c] = rn[c] > tol[c] && it[c] < cap(c) && std::isfinite(rn[c]);
        }
    }
    return finish(B, out, "viscous", it, r0, rn, bnorm, tol);
  }

  int step(hbf_batch* B, hbf_step_stats* stats) override {
    const int n = B->ncav;
    std::vector<hbf_solve_stats> smac(n), svisc(n), snod(n);
    const int* all = B->mask_all;
    int worst = HBF_OK, st;
    auto keep = [&](int s) {
      if (s == HBF_ERR_NOT_CONVERGED) {
        if (worst == HBF_OK) worst = s;
        return false;
      }
      return s != HBF_OK;
    };
    auto mark = [&](int q) {
      if (B->prof) cudaEventRecord(B->pev[q], B->stream);
    };
    mark(0);
    st = replay(B, g_pre, [&] {
      explicit_stage(B, B->expl, 0);
      run<OpTensorLu<D>>(B, tlu, B->H[0][kCells], all);
      explicit_stage(B, B->expl, 1);
      run<OpZero<double>>(B, zero_phi, B->H[0][kCells], all);
      prep_visc(B);
    });
    if (st) return st;
    mark(1);
    if (keep(st = mg_solve(B, 0, smac.data()))) return st;
    mark(2);
    st = replay(B, g_post, [&] {
      explicit_stage(B, B->expl, 2);
      run<OpCopy<double>>(B, cp_in, B->H[0][kCellsD], all);
    });
    if (st) return st;
    mark(3);
    if (keep(st = visc_solve(B, svisc.data()))) return st;
    mark(4);
    if ((st = replay(B, g_nrhs, [&] { explicit_stage(B, B->expl, 3); }))) return st;
    mark(5);
    if (keep(st = mg_solve(B, 1, snod.data()))) return st;
    mark(6);
    st = replay(B, g_upd, [&] {
      explicit_stage(B, B->expl, 4);
      run<OpCopy<double>>(B, cp_out, B->H[0][kCellsD], all);
    });
    if (st) return st;
    mark(7);
    if (B->prof) {
      if ((st = bcheck(B, cudaEventSynchronize(B->pev[7]), "phase timing"))) return st;
      for (int q = 0; q < 7; ++q) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, B->pev[q], B->pev[q + 1]);
        B->phase_ms[q] += ms;
      }
      ++B->prof_steps;
    }
    if (stats)
      for (int c = 0; c < n; ++c) {
        stats[c].mac = smac[c];
        stats[c].visc = svisc[c];
        stats[c].nodal = snod[c];
      }
    if ((st = bcheck(B, cudaGetLastError(), "batched step"))) return st;
    return worst;
  }

  int probe(hbf_batch* B) override {
    int st = replay(B, g_pre, [&] {
      const int* all = B->mask_all;
      explicit_stage(B, B->expl, 0);
      run<OpTensorLu<D>>(B, tlu, B->H[0][kCells], all);
      explicit_stage(B, B->expl, 1);
      run<OpZero<double>>(B, zero_phi, B->H[0][kCells], all);
      prep_visc(B);
    });
    if (st) return st;
    set_mask(B, std::vector<char>(B->ncav, 1));
    return vcyc(B, vph);
  }
};

}  // namespace batch
}  // namespace hb

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
using namespace hb;
using namespace hb::batch;

namespace {

Sig sig_of(hbf_batch* B, int c) {
  hbf_ctx* x = B->cav[c];
  Sig s;
  std::memset(&s, 0, sizeof s);
  s.rheo = x->rheo;
  s.rho = x->rho;
  for (int a = 0; a < 3; ++a) s.f[a] = x->f[a];
  s.dt = B->dt[c];
  s.pv = x->predictor_visc;
  s.cfg = x->cfg;
  s.u = x->u;
  s.ustar = x->ustar;
  s.p = x->p;
  s.walls_version = x->walls_version;
  s.theta = x->theta;
  return s;
}

bool sig_eq(const Sig& a, const Sig& b) {
  return a.rheo.c2 == b.rheo.c2 && a.rheo.n == b.rheo.n && a.rheo.tau == b.rheo.tau && a.rheo.m == b.rheo.m &&
         a.rheo.reg_power == b.rheo.reg_power && a.rho == b.rho && a.f[0] == b.f[0] && a.f[1] == b.f[1] &&
         a.f[2] == b.f[2] && a.dt == b.dt && a.pv == b.pv && a.cfg.rtol == b.cfg.rtol &&
         a.cfg.max_cycles == b.cfg.max_cycles && a.cfg.nu1 == b.cfg.nu1 && a.cfg.nu2 == b.cfg.nu2 &&
         a.cfg.nu_bottom == b.cfg.nu_bottom && a.u == b.u && a.ustar == b.ustar && a.p == b.p &&
         a.walls_version == b.walls_version && a.theta == b.theta;
}

void release_prepared(hbf_batch* B) {
  if (B->stream) cudaStreamSynchronize(B->stream);
  delete B->sol;
  B->sol = nullptr;
  if (B->expl) explicit_destroy(B->expl);
  B->expl = nullptr;
  for (void* p : B->tables) cudaFree(p);
  B->tables.clear();
  for (void* p : B->lallocs) cudaFree(p);
  B->lallocs.clear();
  B->part = nullptr;
  for (int l = 0; l < kMaxLev; ++l)
    for (int s = 0; s < kSpaces; ++s) {
      B->H[l][s] = List();
      B->A[l][s] = List();
    }
  B->prepared = false;
}

// lists, tables and exact bottom inverses for the current settings
int prepare(hbf_batch* B) {
  release_prepared(B);
  const SolverCfg& c0 = B->cav[0]->cfg;
  B->maxlev = 0;
  B->nlev.assign(B->ncav, 0);
  for (int c = 0; c < B->ncav; ++c) {
    hbf_ctx* x = B->cav[c];
    if (!(B->dt[c] > 0.0)) return bfail(B, HBF_ERR_ARG, "every cavity needs a positive time step (hbf_batch_set_dt)");
    if (x->cfg.nu1 != c0.nu1 || x->cfg.nu2 != c0.nu2)
      return bfail(B, HBF_ERR_ARG, "all cavities of a batch need the same smoothing counts nu1, nu2");
    if (x->g.per[0] || x->g.per[1] || x->g.per[2])
      return bfail(B, HBF_ERR_ARG, "the batched sweep has walls on every face (no periodic axes)");
    B->nlev[c] = (int)x->lv.size();
    if (B->nlev[c] > kMaxLev) return bfail(B, HBF_ERR_ARG, "too many multigrid levels");
    B->maxlev = std::max(B->maxlev, B->nlev[c]);
    const Geom& g = x->lv.back().g;
    if ((long long)B->dim * g.ncell > kDenseMax || g.nnode + 0LL > kDenseMax) {
      char buf[160];
      snprintf(buf, sizeof buf, "cavity %d coarsens only to %d x %d x %d cells: the batched sweep needs an exact "
               "bottom solve (at most %d unknowns)", c, g.n[0], g.n[1], g.n[2], kDenseMax);
      return bfail(B, HBF_ERR_ARG, buf);
    }
    ensure_dense(x, 1, 0.0);
    ensure_dense(x, 2, 0.0);
  }
  B->tail_level = B->maxlev;
  if (B->tail_cells > 0)
    for (int l = 0; l < B->maxlev; ++l) {
      bool small = true;
      for (int c = 0; c < B->ncav && small; ++c)
        if (l < B->nlev[c]) small = B->cav[c]->lv[l].g.ncell <= B->tail_cells;
      if (small) {
        B->tail_level = l;
        break;
      }
    }
  int st = B->dim == 2 ? build_lists<2>(B) : build_lists<3>(B);
  if (st) return st;
  void* part = nullptr;
  if (cudaMalloc(&part, sizeof(double) * std::max(B->max_tiles, 1)) != cudaSuccess)
    return bfail(B, HBF_ERR_OOM, "partials");
  B->lallocs.push_back(part);
  B->part = (double*)part;
  B->expl = explicit_create(B);
  if (B->dim == 2) {
    if (B->precision == HBF_MIXED) {
      auto* s = new SolversT<2, float>();
      B->sol = s;
      s->build(B);
    } else {
      auto* s = new SolversT<2, double>();
      B->sol = s;
      s->build(B);
    }
  } else {
    if (B->precision == HBF_MIXED) {
      auto* s = new SolversT<3, float>();
      B->sol = s;
      s->build(B);
    } else {
      auto* s = new SolversT<3, double>();
      B->sol = s;
      s->build(B);
    }
  }
  B->sig.resize(B->ncav);
  for (int c = 0; c < B->ncav; ++c) B->sig[c] = sig_of(B, c);
  B->act_uploaded.clear();
  st = bcheck(B, cudaStreamSynchronize(B->stream), "batch preparation");
  if (st) return st;
  st = bcheck(B, cudaGetLastError(), "batch preparation");
  if (st) return st;
  B->prepared = true;
  return HBF_OK;
}

int ensure_prepared(hbf_batch* B) {
  bool ok = B->prepared && (int)B->sig.size() == B->ncav;
  for (int c = 0; c < B->ncav && ok; ++c) ok = sig_eq(B->sig[c], sig_of(B, c));
  return ok ? HBF_OK : prepare(B);
}

template <typename T>
int dalloc(hbf_batch* B, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) return bfail(B, HBF_ERR_OOM, "batch allocation");
  B->allocs.push_back(q);
  *p = (T*)q;
  return HBF_OK;
}

}  // namespace

extern "C" {

int hbf_batch_create(hbf_batch** out, int dim, int ncav, const int64_t* n, const double* h, const double* wall_u,
                     int precision, void* stream) {
  if (!out) return HBF_ERR_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || ncav < 1 || !n || !h) return HBF_ERR_ARG;
  if (precision != HBF_FP64 && precision != HBF_MIXED) return HBF_ERR_ARG;
  auto* B = new (std::nothrow) hbf_batch();
  if (!B) return HBF_ERR_OOM;
  B->dim = dim;
  B->ncav = ncav;
  B->precision = precision;
  B->stream = (cudaStream_t)stream;
  if (!B->stream) {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete B;
      return HBF_ERR_CUDA;
    }
    B->own_stream = true;
  }
  B->dt.assign(ncav, 0.0);
  int st = HBF_OK;
  for (int c = 0; c < ncav && !st; ++c) {
    hbf_ctx* x = nullptr;
    st = hbf_init_grid(&x, dim, n + 3 * (size_t)c, h[c], wall_u ? wall_u + 18 * (size_t)c : nullptr, precision,
                       (void*)B->stream);
    if (!st) B->cav.push_back(x);
  }
  if (!st) st = dalloc(B, &B->mask_all, ncav);
  if (!st) st = dalloc(B, &B->mask_act, ncav);
  if (!st) st = dalloc(B, &B->red, (size_t)kRedSlots * ncav);
  if (!st) st = dalloc(B, &B->scal, (size_t)4 * ncav);
  if (!st && cudaMallocHost((void**)&B->h_act, sizeof(int) * ncav) != cudaSuccess) st = HBF_ERR_OOM;
  if (!st && cudaMallocHost((void**)&B->hred, sizeof(double) * kRedSlots * ncav) != cudaSuccess) st = HBF_ERR_OOM;
  if (!st && cudaMallocHost((void**)&B->hscal, sizeof(double) * 4 * ncav) != cudaSuccess) st = HBF_ERR_OOM;
  if (!st) {
    std::vector<int> ones(ncav, 1);
    if (cudaMemcpy(B->mask_all, ones.data(), sizeof(int) * ncav, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->mask_act, ones.data(), sizeof(int) * ncav, cudaMemcpyHostToDevice) != cudaSuccess)
      st = HBF_ERR_CUDA;
    std::memset(B->hscal, 0, sizeof(double) * 4 * ncav);
  }
  if (st) {
    hbf_batch_destroy(B);
    return st;
  }
  *out = B;
  return HBF_OK;
}

void hbf_batch_destroy(hbf_batch* B) {
  if (!B) return;
  release_prepared(B);
  for (hbf_ctx* x : B->cav) hbf_destroy(x);
  for (void* p : B->allocs) cudaFree(p);
  if (B->h_act) cudaFreeHost(B->h_act);
  if (B->hred) cudaFreeHost(B->hred);
  if (B->hscal) cudaFreeHost(B->hscal);
  for (int q = 0; q < 8; ++q)
    if (B->pev[q]) cudaEventDestroy(B->pev[q]);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

int hbf_batch_cavity(hbf_batch* B, int i, hbf_ctx** ctx) {
  if (!B || !ctx || i < 0 || i >= B->ncav) return HBF_ERR_ARG;
  *ctx = B->cav[i];
  return HBF_OK;
}

int hbf_batch_set_dt(hbf_batch* B, const double* dt) {
  if (!B || !dt) return HBF_ERR_ARG;
  for (int c = 0; c < B->ncav; ++c)
    if (!(dt[c] > 0.0)) return bfail(B, HBF_ERR_ARG, "dt must be positive");
  for (int c = 0; c < B->ncav; ++c) B->dt[c] = dt[c];
  return HBF_OK;
}

int hbf_batch_set_tiling(hbf_batch* B, int tile, int blocks_per_sm) {
  if (!B || tile < 32 || tile > (1 << 24) || blocks_per_sm < 1 || blocks_per_sm > 64) return HBF_ERR_ARG;
  if (tile != B->tile || blocks_per_sm != B->blocks_per_sm) {
    release_prepared(B);
    B->tile = tile;
    B->blocks_per_sm = blocks_per_sm;
  }
  return HBF_OK;
}

int hbf_batch_set_tail(hbf_batch* B, int max_cells) {
  if (!B || max_cells < 0) return HBF_ERR_ARG;
  if (max_cells != B->tail_cells) {
    release_prepared(B);
    B->tail_cells = max_cells;
  }
  return HBF_OK;
}

int hbf_batch_get_tiling(const hbf_batch* B, int* tile, int* blocks_per_sm, int64_t* tiles_level0) {
  if (!B) return HBF_ERR_ARG;
  if (tile) *tile = B->tile;
  if (blocks_per_sm) *blocks_per_sm = B->blocks_per_sm;
  if (tiles_level0) *tiles_level0 = B->prepared ? B->H[0][kCells].n : 0;
  return HBF_OK;
}

int hbf_batch_step(hbf_batch* B, hbf_step_stats* stats) {
  if (!B) return HBF_ERR_ARG;
  int st = ensure_prepared(B);
  if (st) return st;
  st = B->sol->step(B, stats);
  if (st == HBF_OK || st == HBF_ERR_NOT_CONVERGED)
    for (int c = 0; c < B->ncav; ++c) {
      B->cav[c]->t += B->dt[c];
      ++B->cav[c]->nstep;
      B->cav[c]->prev_valid = false;  // the batch keeps no copy of u^m
    }
  return st;
}

int hbf_batch_autotune(hbf_batch* B, int reps, int* best_tile, int* best_bps, double* best_ms) {
  if (!B || reps < 1) return HBF_ERR_ARG;
  static const int tiles[] = {1024, 2048, 4096, 8192};
  static const int bpss[] = {4, 8, 16};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = INFINITY;
  int bt = B->tile, bb = B->blocks_per_sm;
  int st = HBF_OK;
  for (int tile : tiles) {
    for (int bps : bpss) {
      if ((st = hbf_batch_set_tiling(B, tile, bps))) break;
      if ((st = prepare(B))) break;
      if ((st = B->sol->probe(B))) break;  // warm-up and graph capture
      cudaEventRecord(e0, B->stream);
      for (int r = 0; r < reps && !st; ++r) st = B->sol->probe(B);
      cudaEventRecord(e1, B->stream);
      if (st || (st = bcheck(B, cudaEventSynchronize(e1), "autotune"))) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = (double)ms / reps;
      if (per < best) {
        best = per;
        bt = tile;
        bb = bps;
      }
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if ((st = hbf_batch_set_tiling(B, bt, bb))) return st;
  if ((st = prepare(B))) return st;
  if (best_tile) *best_tile = bt;
  if (best_bps) *best_bps = bb;
  if (best_ms) *best_ms = best;
  return HBF_OK;
}

int hbf_batch_profile(hbf_batch* B, int on) {
  if (!B) return HBF_ERR_ARG;
  int st = bcheck(B, cudaStreamSynchronize(B->stream), "profile");
  if (st) return st;
  if (on && !B->pev[0])
    for (int q = 0; q < 8; ++q)
      if ((st = bcheck(B, cudaEventCreate(&B->pev[q]), "profile events"))) return st;
  B->prof = on != 0;
  for (int q = 0; q < 7; ++q) B->phase_ms[q] = 0.0;
  for (int q = 0; q < 3; ++q) B->trips[q] = 0;
  B->prof_steps = 0;
  return HBF_OK;
}

int hbf_batch_profile_read(const hbf_batch* B, double phase_ms[7], int64_t trips[3], int64_t* steps) {
  if (!B) return HBF_ERR_ARG;
  if (phase_ms)
    for (int q = 0; q < 7; ++q) phase_ms[q] = B->phase_ms[q];
  if (trips)
    for (int q = 0; q < 3; ++q) trips[q] = B->trips[q];
  if (steps) *steps = B->prof_steps;
  return HBF_OK;
}

int64_t hbf_batch_launch_count(const hbf_batch* B) { return B ? (int64_t)B->nlaunch : HBF_ERR_ARG; }

const char* hbf_batch_last_error(const hbf_batch* B) { return B ? B->err.c_str() : "null batch"; }

int hbf_batch_sync(hbf_batch* B) {
  if (!B) return HBF_ERR_ARG;
  return bcheck(B, cudaStreamSynchronize(B->stream), "hbf_batch_sync");
}

}  // extern "C"
