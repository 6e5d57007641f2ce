// Shared device-side definitions of the GB300 step library: grid geometry,
// indexing, wall ghosts and small helpers.  Every kernel is templated on the
// space dimension D (2 or 3); for D == 2 the z extent is 1 and z loops vanish.
//
// Memory layout (HBM): structure of arrays, x fastest.
//   cell field, component c:   base + c*ncell + i + nx*(j + ny*k)
//   a-face field, component c: base + c*nface[a] + i + (nx+da)*(j + (ny+db)*k)
//                              (one extra point along a)
//   node field:                i + (nx+1)*(j + (ny+1)*k)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hb {

constexpr int kThreads = 256;

struct Geom {
  int n[3];          // cells per axis (n[2] == 1 in 2D)
  double h;          // cell size (equal on all axes)
  double wu[3][2][3];  // wall velocity [axis][side][component]
  int ncell;
  int nnode;
  int nface[3];
};

struct Rheo {
  double c2;     // 2^(n-1) K
  double n;      // flow index
  double tau;    // yield stress tau_y
  double m;      // Papanastasiou exponent 1/epsilon
  int reg_power; // 1: regularise the whole bracket (Eq. 23); 0: yield term only
};

template <int D>
__host__ __device__ inline int cidx(const Geom& g, int i, int j, int k) {
  return i + g.n[0] * (j + g.n[1] * k);
}

__host__ __device__ inline int nidx(const Geom& g, int i, int j, int k) {
  return i + (g.n[0] + 1) * (j + (g.n[1] + 1) * k);
}

// index of a face normal to axis a with lower-corner cell index (i, j, k)
__host__ __device__ inline int fidx(const Geom& g, int a, int i, int j, int k) {
  int ex = g.n[0] + (a == 0), ey = g.n[1] + (a == 1);
  return i + ex * (j + ey * k);
}

template <int D>
__host__ __device__ inline void cell_coords(const Geom& g, int t, int& i, int& j, int& k) {
  i = t % g.n[0];
  int r = t / g.n[0];
  if (D == 3) {
    j = r % g.n[1];
    k = r / g.n[1];
  } else {
    j = r;
    k = 0;
  }
}

// Velocity component c at cell (i,j,k) where at most one axis is out of range
// by one or two cells: odd reflection about the wall value of that face,
// g = 2 u_b - u_mirror (homogeneous: u_b = 0).
template <int D, typename T>
__host__ __device__ inline T uget(const T* __restrict__ uc, const Geom& g, int c, int i, int j, int k,
                                  bool hom) {
  // the first out-of-range axis (x, then y, then z) selects the reflection
  int ax = -1, side = 0;
  if (i < 0) {
    ax = 0; side = 0; i = -i - 1;
  } else if (i >= g.n[0]) {
    ax = 0; side = 1; i = 2 * g.n[0] - 1 - i;
  } else if (j < 0) {
    ax = 1; side = 0; j = -j - 1;
  } else if (j >= g.n[1]) {
    ax = 1; side = 1; j = 2 * g.n[1] - 1 - j;
  } else if (D == 3 && k < 0) {
    ax = 2; side = 0; k = -k - 1;
  } else if (D == 3 && k >= g.n[2]) {
    ax = 2; side = 1; k = 2 * g.n[2] - 1 - k;
  }
  T v = uc[cidx<D>(g, i, j, k)];
  if (ax < 0) return v;
  T ub = hom ? T(0) : T(g.wu[ax][side][c]);
  return T(2) * ub - v;
}

// Scalar with even reflection across walls (Neumann ghosts; one layer).
template <int D, typename T>
__host__ __device__ inline T nget(const T* __restrict__ x, const Geom& g, int i, int j, int k) {
  i = i < 0 ? -i - 1 : (i >= g.n[0] ? 2 * g.n[0] - 1 - i : i);
  j = j < 0 ? -j - 1 : (j >= g.n[1] ? 2 * g.n[1] - 1 - j : j);
  if (D == 3) k = k < 0 ? -k - 1 : (k >= g.n[2] ? 2 * g.n[2] - 1 - k : k);
  return x[cidx<D>(g, i, j, k)];
}

// Node value with even reflection across walls (node -1 -> 1, n+1 -> n-1).
template <int D, typename T>
__host__ __device__ inline T ndget(const T* __restrict__ x, const Geom& g, int i, int j, int k) {
  i = i < 0 ? -i : (i > g.n[0] ? 2 * g.n[0] - i : i);
  j = j < 0 ? -j : (j > g.n[1] ? 2 * g.n[1] - j : j);
  if (D == 3) k = k < 0 ? -k : (k > g.n[2] ? 2 * g.n[2] - k : k);
  return x[nidx(g, i, j, k)];
}

template <int D>
__host__ __device__ inline Geom coarse_of(const Geom& f) {
  Geom c = f;
  c.n[0] = f.n[0] / 2;
  c.n[1] = f.n[1] / 2;
  c.n[2] = D == 3 ? f.n[2] / 2 : 1;
  c.h = 2.0 * f.h;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 3; ++q) c.wu[a][s][q] = 0.0;
  c.ncell = c.n[0] * c.n[1] * c.n[2];
  c.nnode = (c.n[0] + 1) * (c.n[1] + 1) * (D == 3 ? c.n[2] + 1 : 1);
  c.nface[0] = (c.n[0] + 1) * c.n[1] * c.n[2];
  c.nface[1] = c.n[0] * (c.n[1] + 1) * c.n[2];
  c.nface[2] = D == 3 ? c.n[0] * c.n[1] * (c.n[2] + 1) : 0;
  return c;
}

inline int grid_for(long long work, int cap = 152 * 16) {
  long long b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace hb
