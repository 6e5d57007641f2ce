// Batched execution over many independent cavities: one persistent launch
// per stage walks a work list of tiles (cavity, element range) with the
// cavity's own arguments, so cavities of different sizes share each launch.
#pragma once
#include "hb_internal.h"

namespace hb {
namespace batch {

constexpr int kMaxLev = 16;  // multigrid levels a batch or a fused tail handles

struct Tile {
  int cav;
  int begin;
  int end;
};

// Persistent grid-stride over tiles; a tile whose cavity is masked off is
// skipped (mask may be null).  Op::apply(arg, element, extra) does the work.
template <class Op>
__global__ void __launch_bounds__(256) k_batch(const typename Op::Arg* __restrict__ args,
                                               const Tile* __restrict__ tiles, int ntiles,
                                               const int* __restrict__ mask, int extra) {
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const Tile T = tiles[ti];
    if (mask && !mask[T.cav]) continue;
    const typename Op::Arg& a = args[T.cav];
    for (int t = T.begin + (int)threadIdx.x; t < T.end; t += (int)blockDim.x) Op::apply(a, t, extra);
  }
}

// face spaces: t runs over the faces of every axis, axis-major; returns the
// axis and leaves t as the index within that axis
__device__ inline int face_axis(const Geom& g, int& t) {
  if (t < g.nface[0]) return 0;
  t -= g.nface[0];
  if (t < g.nface[1]) return 1;
  t -= g.nface[1];
  return 2;
}

// Per-tile partial reductions (mode 0: max |x| with non-finite -> +inf,
// mode 1: sum x, mode 2: sum x*y, mode 3: sum w_node x for nodal arrays);
// a second kernel combines each cavity's contiguous range of tiles in a fixed
// order, so results do not depend on scheduling.  Sums run in FP64 for either
// element type.
template <typename T>
struct RedArg {
  const T* x;
  const T* y;
  Geom g;
  int dim;
};

__host__ __device__ inline double node_weight(const Geom& g, int dim, int t) {
  int i, j, k;
  node_coords(g, t, i, j, k);
  double w = 1.0;
  w = node_weight(g, i, j, k, dim);
  return w;
}

// One warp per tile: lanes stride over the tile's elements, then a fixed
// xor-shuffle tree; no block barriers, so short tiles stay cheap.
template <typename T>
__global__ void __launch_bounds__(256) k_batch_reduce(const RedArg<T>* __restrict__ args,
                                                      const Tile* __restrict__ tiles, int ntiles,
                                                      const int* __restrict__ mask, int mode,
                                                      double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int ti = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); ti < ntiles; ti += nwarps) {
    const Tile T0 = tiles[ti];
    double acc = 0.0;
    if (!mask || mask[T0.cav]) {
      const RedArg<T> a = args[T0.cav];
      // max and dot accumulate in T over the lane's share of the tile (at
      // most tile/32 elements), then in FP64 across lanes and tiles
      if (mode == 0) {
        T m = T(0);
        for (int t = T0.begin + lane; t < T0.end; t += 32) {
          T v = a.x[t] < T(0) ? -a.x[t] : a.x[t];
          if (!isfinite(v)) v = T(INFINITY);
          m = v > m ? v : m;
        }
        acc = (double)m;
      } else if (mode == 1) {
        for (int t = T0.begin + lane; t < T0.end; t += 32) acc += (double)a.x[t];
      } else if (mode == 2) {
        T d = T(0);
        for (int t = T0.begin + lane; t < T0.end; t += 32) d += a.x[t] * a.y[t];
        acc = (double)d;
      } else {
        for (int t = T0.begin + lane; t < T0.end; t += 32) acc += node_weight(a.g, a.dim, t) * (double)a.x[t];
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, acc, off);
      acc = mode == 0 ? fmax(acc, o) : acc + o;
    }
    if (lane == 0) part[ti] = acc;
  }
}

// out[c] = (combination of the partials of cavity c's tiles
// [first[c], first[c+1])) * (scale ? scale[c] : 1); one warp per cavity,
// fixed order
static __global__ void __launch_bounds__(256) k_batch_combine(const double* __restrict__ part,
                                                              const int* __restrict__ first, int ncav, int mode,
                                                              const double* __restrict__ scale,
                                                              double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < ncav; c += nwarps) {
    double s = 0.0;
    for (int q = first[c] + lane; q < first[c + 1]; q += 32) s = mode == 0 ? fmax(s, part[q]) : s + part[q];
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, s, off);
      s = mode == 0 ? fmax(s, o) : s + o;
    }
    if (lane == 0) out[c] = scale ? s * scale[c] : s;
  }
}

}  // namespace batch
}  // namespace hb
