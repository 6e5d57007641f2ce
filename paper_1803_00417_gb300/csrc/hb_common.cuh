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
  int per[3];        // 1: the axis is periodic (no walls normal to it), 0: walls
  double h;          // cell size (equal on all axes)
  double wu[3][2][3];  // wall velocity [axis][side][component]
  int ncell;
  int nnode;
  int nface[3];
  // derived on the host by geom_finish(): the constants 1/h, 1/h^2, 0.25/h,
  // h^2 (and their FP32 roundings), and exact division multipliers for the
  // index decompositions (see divm)
  double ih, ihh, q4, hh;
  float fih, fihh, fq4, fhh;
  float fwu[3][2][3];  // FP32 wall velocities
  unsigned long long m_n0, m_n1, m_e0, m_e1, m_rb, m_mc0[2], m_mc1[2];
  unsigned long long m_rbx, m_xi;    // (n0 - 1) / 2 and n0 - 2: the x-interior cell maps
  unsigned long long m_rbxg, m_xig;  // their row-group sizes 16 M + 32
  unsigned long long m_sx, m_n1i;    // n0 / 2 - 1 and n1 - 2: the colour-split interior map
};

// Multiplier M for the exact quotient t / d = floor(t * M / 2^64) of any
// 0 <= t < 2^32 by a fixed 1 <= d < 2^32: M = ceil(2^64 / d), with the error
// t * (M d - 2^64) / (d 2^64) < 1/d never reaching the next integer.  d = 1
// gives M = 0 (wrapped), handled by divm.
__host__ __device__ inline unsigned long long div_magic(unsigned d) {
  return d <= 1 ? 0ull : (~0ull) / d + 1ull;
}

__host__ __device__ __forceinline__ int divm(int t, int d, unsigned long long M) {
#ifdef __CUDA_ARCH__
  return M ? (int)__umul64hi((unsigned long long)(unsigned)t, M) : t;
#else
  (void)M;
  return t / d;
#endif
}

__host__ __device__ inline void geom_finish(Geom& g) {
  g.ih = 1.0 / g.h;
  g.ihh = 1.0 / (g.h * g.h);
  g.q4 = 0.25 / g.h;
  g.hh = g.h * g.h;
  g.fih = (float)g.ih;
  g.fihh = (float)g.ihh;
  g.fq4 = (float)g.q4;
  g.fhh = (float)g.hh;
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 3; ++q) g.fwu[a][sd][q] = (float)g.wu[a][sd][q];
  g.m_n0 = div_magic((unsigned)g.n[0]);
  g.m_n1 = div_magic((unsigned)g.n[1]);
  g.m_e0 = div_magic((unsigned)(g.n[0] + 1));
  g.m_e1 = div_magic((unsigned)(g.n[1] + 1));
  g.m_rb = div_magic((unsigned)((g.n[0] + 1) / 2));
  g.m_rbx = div_magic((unsigned)((g.n[0] - 1) / 2));
  g.m_xi = div_magic((unsigned)(g.n[0] > 2 ? g.n[0] - 2 : 0));
  g.m_rbxg = div_magic((unsigned)(16 * ((g.n[0] - 1) / 2) + 32));
  g.m_xig = div_magic((unsigned)(16 * (g.n[0] > 2 ? g.n[0] - 2 : 0) + 32));
  g.m_sx = div_magic((unsigned)(g.n[0] >= 4 ? g.n[0] / 2 - 1 : 1));
  g.m_n1i = div_magic((unsigned)(g.n[1] > 2 ? g.n[1] - 2 : 1));
  for (int b = 0; b < 2; ++b) {
    g.m_mc0[b] = div_magic((unsigned)((g.n[0] + 1 - b + 1) / 2));
    g.m_mc1[b] = div_magic((unsigned)((g.n[1] + 1 - b + 1) / 2));
  }
}

// the derived constants in arithmetic T
template <typename T>
__host__ __device__ inline T g_wu(const Geom& g, int a, int s, int c);
template <>
__host__ __device__ inline double g_wu<double>(const Geom& g, int a, int s, int c) { return g.wu[a][s][c]; }
template <>
__host__ __device__ inline float g_wu<float>(const Geom& g, int a, int s, int c) { return g.fwu[a][s][c]; }

template <typename T>
__host__ __device__ inline T g_ih(const Geom& g);
template <>
__host__ __device__ inline double g_ih<double>(const Geom& g) { return g.ih; }
template <>
__host__ __device__ inline float g_ih<float>(const Geom& g) { return g.fih; }
template <typename T>
__host__ __device__ inline T g_ihh(const Geom& g);
template <>
__host__ __device__ inline double g_ihh<double>(const Geom& g) { return g.ihh; }
template <>
__host__ __device__ inline float g_ihh<float>(const Geom& g) { return g.fihh; }
template <typename T>
__host__ __device__ inline T g_q4(const Geom& g);
template <>
__host__ __device__ inline double g_q4<double>(const Geom& g) { return g.q4; }
template <>
__host__ __device__ inline float g_q4<float>(const Geom& g) { return g.fq4; }
template <typename T>
__host__ __device__ inline T g_hh(const Geom& g);
template <>
__host__ __device__ inline double g_hh<double>(const Geom& g) { return g.hh; }
template <>
__host__ __device__ inline float g_hh<float>(const Geom& g) { return g.fhh; }

struct Rheo {
  double c2;     // 2^(n-1) K
  double n;      // flow index
  double tau;    // yield stress tau_y
  double m;      // Papanastasiou exponent 1/epsilon
  int reg_power; // 1: regularise the whole bracket (Eq. 23); 0: yield term only
  int e2;        // twice the power-law exponent (n, or n - 1 without reg_power)
                 // when it is an integer of magnitude <= 8, else kGeneralPow
};

constexpr int kGeneralPow = 1 << 20;

// e2 of a flow index (host side, set with the rheology)
inline int rheo_e2(double n, int reg_power) {
  const double e2 = 2.0 * (reg_power ? n : n - 1.0);
  const double r = (double)(long long)e2;
  return (r == e2 && e2 >= -8.0 && e2 <= 8.0) ? (int)r : kGeneralPow;
}

template <int D>
__host__ __device__ inline int cidx(const Geom& g, int i, int j, int k) {
  return i + g.n[0] * (j + g.n[1] * k);
}

// Cell (i, j, k) of a 3D level with even n0 in the colour-split layout: the
// cells with i + j + k even first, then the odd ones, each half row-major
// over (j, k) with n0 / 2 cells per row (cell i at i / 2).  A red-black sweep
// then reads and writes unit-stride runs of one colour.
__host__ __device__ inline int sidx(const Geom& g, int i, int j, int k) {
  return ((i + j + k) & 1) * (g.ncell >> 1) + (j + g.n[1] * k) * (g.n[0] >> 1) + (i >> 1);
}

// the natural (SP false) or colour-split (SP true, 3D only) cell index
template <int D, bool SP = false>
__host__ __device__ inline int lidx(const Geom& g, int i, int j, int k) {
  return SP ? sidx(g, i, j, k) : cidx<D>(g, i, j, k);
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
  const int r = divm(t, g.n[0], g.m_n0);
  i = t - r * g.n[0];
  if (D == 3) {
    k = divm(r, g.n[1], g.m_n1);
    j = r - k * g.n[1];
  } else {
    j = r;
    k = 0;
  }
}

// node t -> (i, j, k) on the (n0+1) x (n1+1) x (n2+1) node grid
__host__ __device__ inline void node_coords(const Geom& g, int t, int& i, int& j, int& k) {
  const int e0 = g.n[0] + 1, e1 = g.n[1] + 1;
  const int r = divm(t, e0, g.m_e0);
  i = t - r * e0;
  k = divm(r, e1, g.m_e1);
  j = r - k * e1;
}

// a-face t -> (i, j, k) on the face grid (one more point along a)
__host__ __device__ inline void face_coords(const Geom& g, int a, int t, int& i, int& j, int& k) {
  const int ex = g.n[0] + (a == 0), ey = g.n[1] + (a == 1);
  const int r = divm(t, ex, a == 0 ? g.m_e0 : g.m_n0);
  i = t - r * ex;
  k = divm(r, ey, a == 1 ? g.m_e1 : g.m_n1);
  j = r - k * ey;
}

// A periodic axis: a cell index within one period of [0, n) wrapped into it;
// a node index within one period of [0, n] wrapped into it (node n is the
// copy of node 0, kept so that nodal arrays have n+1 points on every axis).
__host__ __device__ inline int wrap_cell(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__host__ __device__ inline int wrap_node(int i, int n) { return i < 0 ? i + n : (i > n ? i - n : i); }

// Weight of node (i, j, k) in the mean of a nodal field: the fraction of its
// dual cell inside the domain (1/2 per wall axis on which the node lies on
// the wall), 0 for the copy node n on a periodic axis (so that every distinct
// node counts once)
__host__ __device__ inline double node_weight(const Geom& g, int i, int j, int k, int dim) {
  const int p[3] = {i, j, k};
  double w = 1.0;
  for (int a = 0; a < dim; ++a) {
    if (g.per[a]) {
      if (p[a] == g.n[a]) w = 0.0;
    } else if (p[a] == 0 || p[a] == g.n[a]) {
      w *= 0.5;
    }
  }
  return w;
}

// Velocity component c at cell (i,j,k) where at most one axis is out of range
// by one or two cells: odd reflection about the wall value of that face,
// g = 2 u_b - u_mirror (homogeneous: u_b = 0).
template <int D, typename T>
__host__ __device__ inline T uget(const T* __restrict__ uc, const Geom& g, int c, int i, int j, int k,
                                  bool hom) {
  // periodic axes wrap; then the first out-of-range axis (x, then y, then z)
  // selects the reflection
  if (g.per[0]) i = wrap_cell(i, g.n[0]);
  if (g.per[1]) j = wrap_cell(j, g.n[1]);
  if (D == 3 && g.per[2]) k = wrap_cell(k, g.n[2]);
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
  T ub = hom ? T(0) : g_wu<T>(g, ax, side, c);
  return T(2) * ub - v;
}

// Scalar with even reflection across walls (Neumann ghosts; one layer),
// wrapped on periodic axes.
template <int D, typename T>
__host__ __device__ inline T nget(const T* __restrict__ x, const Geom& g, int i, int j, int k) {
  if (g.per[0]) i = wrap_cell(i, g.n[0]);
  if (g.per[1]) j = wrap_cell(j, g.n[1]);
  if (D == 3 && g.per[2]) k = wrap_cell(k, g.n[2]);
  i = i < 0 ? -i - 1 : (i >= g.n[0] ? 2 * g.n[0] - 1 - i : i);
  j = j < 0 ? -j - 1 : (j >= g.n[1] ? 2 * g.n[1] - 1 - j : j);
  if (D == 3) k = k < 0 ? -k - 1 : (k >= g.n[2] ? 2 * g.n[2] - 1 - k : k);
  return x[cidx<D>(g, i, j, k)];
}

// Node value with even reflection across walls (node -1 -> 1, n+1 -> n-1),
// wrapped on periodic axes (node -1 -> n-1, n+1 -> 1).
// PER = false compiles the wraps out (a level with walls on every axis).
template <int D, typename T, bool PER = true>
__host__ __device__ inline T ndget(const T* __restrict__ x, const Geom& g, int i, int j, int k) {
  if (PER) {
    if (g.per[0]) i = wrap_node(i, g.n[0]);
    if (g.per[1]) j = wrap_node(j, g.n[1]);
    if (D == 3 && g.per[2]) k = wrap_node(k, g.n[2]);
  }
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
  geom_finish(c);
  return c;
}

inline int grid_for(long long work, int cap = 152 * 16) {
  long long b = (work + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace hb
