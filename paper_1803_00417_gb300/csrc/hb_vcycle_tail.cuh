// Argument records of the multigrid operations on one cavity's level, the
// block-level exact bottom solve, and the fused V-cycle tail: one thread block
// walks a cavity's small levels (smoothing, residual, restriction, bottom
// solve, prolongation) with block barriers between the phases.  Used by the
// batched sweep (one block per cavity) and by the single-cavity solves (one
// block).
#pragma once
#include "hb_batch.cuh"
#include "hb_mg_kernels.cuh"

namespace hb {
namespace batch {

enum Kind { kVisc = 0, kMac = 1, kNodal = 2 };

template <typename T>
struct ViscArg {
  T* x;
  const T* b;
  T* out;
  const T* ef[3];
  Geom g;
  T beta;
  int hom;
};

template <typename T>
struct PoisArg {
  T* x;
  T* b;
  T* r;
  Geom g;
};

// grid transfers: restriction writes the coarse right-hand side and zeroes
// the coarse iterate; prolongation adds the coarse correction
template <typename T>
struct XferArg {
  const T* src;
  T* dst;
  T* zero;
  Geom gf, gc;
  int ncomp;
  int sign;
};

template <typename T>
struct BottomArg {
  const double* Minv;
  int m;      // matrix size (n, or n + 1 when bordered)
  int n;      // unknowns
  T* x;
  T* b;
  Geom g;
  int kind;   // 0 viscous, 1 MAC, 2 nodal
  int level;  // the cavity's coarsest level
};

// weighted mean of v over the unknowns of a singular problem, one thread,
// fixed order (n is at most kDenseMax)
template <int D>
__device__ inline double bottom_mean(const double* v, int n, int kind, const Geom& g) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (kind == 2 ? node_weight(g, D, i) : 1.0) * v[i];
  const double wsum = kind == 2 ? (double)g.n[0] * g.n[1] * (D == 3 ? g.n[2] : 1) : (double)n;
  return s * (1.0 / wsum);
}

// exact solve of one cavity's coarsest level by the whole block
template <int D, typename T>
__device__ void bottom_block(const BottomArg<T>& a) {
  __shared__ double sb[kDenseMax + 1];
  __shared__ double sx[kDenseMax + 1];
  __shared__ double mean;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) sb[i] = (double)a.b[i];
  __syncthreads();
  if (a.kind != 0) {
    if (threadIdx.x == 0) mean = bottom_mean<D>(sb, a.n, a.kind, a.g);
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) sb[i] -= mean;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < a.n; ++j) acc += a.Minv[(size_t)i * a.m + j] * sb[j];
    sx[i] = acc;
  }
  __syncthreads();
  if (a.kind != 0) {
    if (threadIdx.x == 0) mean = bottom_mean<D>(sx, a.n, a.kind, a.g);
    __syncthreads();
    for (int i = threadIdx.x; i < a.n; i += blockDim.x) sx[i] -= mean;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) a.x[i] = (T)sx[i];
  __syncthreads();
}

// the argument tables of an instance, by level, for the fused tail kernel
struct TailTabs {
  const void* lv[kMaxLev];
  const void* re[kMaxLev];
  const void* pr[kMaxLev];
  const void* bot;
};

// ---------------------------------------------------------------------------
// fused tail of the V-cycle: one block per cavity runs every level from lf
// down to the cavity's coarsest and back, with block barriers between the
// colour sweeps instead of kernel boundaries.  Same operations in the same
// order as the level-by-level launches; the small levels of all cavities then
// cost one launch per V-cycle instead of about twenty per level.
// ---------------------------------------------------------------------------
template <int D, typename T, int C, bool PER>
__device__ __forceinline__ void tail_visc_colours(const ViscArg<T>& a) {
  const int nt = rb_count<D>(a.g);
  for (int col = 0; col < 2; ++col) {
    for (int t = threadIdx.x; t < nt; t += blockDim.x)
      k_visc_smooth_c_at<D, T, C, PER>(a.x, a.b, a.ef[0], a.ef[1], a.ef[2], a.g, col, a.beta, a.hom, t);
    __syncthreads();
  }
}

template <int D, typename T, int KIND, bool PER>
__device__ __forceinline__ void tail_smooth(const TailTabs& tb, int l, int c) {
  if (KIND == kVisc) {
    const ViscArg<T>& a = ((const ViscArg<T>*)tb.lv[l])[c];
    tail_visc_colours<D, T, 0, PER>(a);
    tail_visc_colours<D, T, 1, PER>(a);
    if (D == 3) tail_visc_colours<D, T, (D == 3 ? 2 : 0), PER>(a);
  } else if (KIND == kMac) {
    const PoisArg<T>& a = ((const PoisArg<T>*)tb.lv[l])[c];
    const int nt = rb_count<D>(a.g);
    for (int col = 0; col < 2; ++col) {
      for (int t = threadIdx.x; t < nt; t += blockDim.x) k_cell_smooth_at<D, T, PER>(a.x, a.b, a.g, col, t);
      __syncthreads();
    }
  } else {
    const PoisArg<T>& a = ((const PoisArg<T>*)tb.lv[l])[c];
    for (int col = 0; col < (1 << D); ++col) {
      const int nt = mc_count<D>(a.g, col);
      for (int t = threadIdx.x; t < nt; t += blockDim.x) k_nodal_smooth_at<D, T, PER>(a.x, a.b, a.g, col, t);
      __syncthreads();
    }
  }
}

// PER = false: every level of every cavity has walls on every axis
template <int D, typename T, int KIND, bool PER = true>
__global__ void __launch_bounds__(256) k_vcycle_tail(TailTabs tb, int lf, int ncav,
                                                           const int* __restrict__ mask, int nu1, int nu2) {
  const int c = blockIdx.x;
  if (c >= ncav || (mask && !mask[c])) return;
  const BottomArg<T>& bot = ((const BottomArg<T>*)tb.bot)[c];
  const int L = bot.level;
  if (L < lf) return;
  for (int l = lf; l < L; ++l) {
    for (int s = 0; s < nu1; ++s) tail_smooth<D, T, KIND, PER>(tb, l, c);
    if (KIND == kVisc) {
      const ViscArg<T>& a = ((const ViscArg<T>*)tb.lv[l])[c];
      for (int t = threadIdx.x; t < a.g.ncell; t += blockDim.x)
        k_visc_op_at<D, T, PER>(a.x, a.b, a.out, a.ef[0], a.ef[1], a.ef[2], a.g, a.beta, a.hom, t);
    } else {
      const PoisArg<T>& a = ((const PoisArg<T>*)tb.lv[l])[c];
      if (KIND == kMac)
        for (int t = threadIdx.x; t < a.g.ncell; t += blockDim.x) k_cell_resid_at<D, T, PER>(a.x, a.b, a.r, a.g, t);
      else
        for (int t = threadIdx.x; t < a.g.nnode; t += blockDim.x) k_nodal_resid_at<D, T, PER>(a.x, a.b, a.r, a.g, t);
    }
    __syncthreads();
    const XferArg<T>& r = ((const XferArg<T>*)tb.re[l])[c];
    if (KIND == kNodal) {
      for (int t = threadIdx.x; t < r.gc.nnode; t += blockDim.x) {
        k_restrict_nodes_at<D, T, PER>(r.src, r.dst, r.gf, r.gc, t);
        r.zero[t] = T(0);
      }
    } else {
      const int n = r.ncomp * r.gc.ncell;
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        k_restrict_cells_at<D, T>(r.src, r.dst, r.gf, r.gc, r.ncomp, t);
        r.zero[t] = T(0);
      }
    }
    __syncthreads();
  }
  bottom_block<D, T>(bot);
  for (int l = L - 1; l >= lf; --l) {
    const XferArg<T>& q = ((const XferArg<T>*)tb.pr[l])[c];
    if (KIND == kNodal) {
      for (int t = threadIdx.x; t < q.gf.nnode; t += blockDim.x) k_prolong_nodes_add_at<D, T>(q.dst, q.src, q.gf, q.gc, t);
    } else {
      const int n = q.ncomp * q.gf.ncell;
      for (int t = threadIdx.x; t < n; t += blockDim.x)
        k_prolong_cells_add_at<D, T, PER>(q.dst, q.src, q.gf, q.gc, q.ncomp, T(q.sign), t);
    }
    __syncthreads();
    for (int s = 0; s < nu2; ++s) tail_smooth<D, T, KIND, PER>(tb, l, c);
  }
}

}  // namespace batch
}  // namespace hb
