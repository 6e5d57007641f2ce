// Colour-split layout of the FP32 finest level of the mixed viscous solve (3D,
// walls on every axis, even n0): its kernels on arrays indexed by sidx
// (hb_common.cuh), each component's cells with i + j + k even first, then the
// odd ones.  A red-black sweep of one colour then reads the other colour's
// half of u_c and writes its own, both unit-stride, and reads b_c of its own
// colour only: none of the opposite colour's bytes of u_c and b_c that every
// 32-byte sector of the natural layout carries along.  The arithmetic is that
// of the natural-layout kernels (visc_gs_core and tensor_core on the same
// gathered values; at wall cells visc_gs_point's and mg_tensor_point's
// operations in the same order; the same transfers through lidx), so both
// layouts give the same values bit for bit.
#pragma once
#include "hb_mg_kernels.cuh"

namespace hb {

// Thread -> cell map of the split kernels: one thread per cell, no loop.
// Block (seg, j, k), j < n1, takes W slots (a multiple of 32, at most 256) of
// row (j, k) per colour, from slot seg W on: the cells i = 2 ih + q with
// ih = m + 1 - q for slots m < n0 / 2 - 1, which leave out the x-wall cell of
// the colour (i = 0 or n0 - 1); they are interior cells unless j or k is on a
// wall.  The blocks (0, n1 + G, k) take the x-wall cells of rows 32 G ..
// 32 G + 31 of plane k, one warp per colour, so that the wall cells run 32 to
// a warp, in blocks dispatched right after their plane's rows (blocks go
// through the grid x, then y, then z), while the rows around them are in L2.
struct SplitMap {
  int W, nseg;
};

__host__ __device__ inline SplitMap split_map(const Geom& g) {
  const int m = (g.n[0] >> 1) - 1;
  int W = (m + 31) / 32 * 32;
  if (W > 256) W = 256;
  return {W, (m + W - 1) / W};
}

// grid and block of a launch over ncol colours
inline dim3 split_grid(const Geom& g) {
  return dim3((unsigned)split_map(g).nseg, (unsigned)(g.n[1] + (g.n[1] + 31) / 32), (unsigned)g.n[2]);
}
inline dim3 split_block_dim(const Geom& g, int ncol) { return dim3((unsigned)(ncol * split_map(g).W), 1, 1); }

// Thread tid of block (seg, jy, k) of a launch over NCOL colours (colour col0
// when NCOL == 1; colour 0 for threads [0, W), colour 1 for [W, 2W) when
// NCOL == 2; in an x-wall block, warp c takes colour c): f(p, P, col,
// interior) for its cell p of colour col at position P of the colour's half
// (P = (j + n1 k) n0 / 2 + i / 2); nothing for a thread without a cell.
template <int NCOL, typename F>
__host__ __device__ __forceinline__ void split_thread(const Geom& g, int col0, int W, int seg, int jy, int k, int tid,
                                                      F&& f) {
  const int hn = g.n[0] >> 1;
  if (jy < g.n[1]) {
    const int j = jy;
    const int col = NCOL == 2 ? (tid >= W ? 1 : 0) : col0;
    const int m = seg * W + tid - (NCOL == 2 && tid >= W ? W : 0);
    if (m >= hn - 1) return;
    const int q = (j + k + col) & 1;  // x parity of the colour's cells in this row
    const int ih = m + 1 - q;
    const int p[3] = {2 * ih + q, j, k};
    const int P = (j + g.n[1] * k) * hn + ih;
    if (j > 0 && j < g.n[1] - 1 && k > 0 && k < g.n[2] - 1)
      f(p, P, col, true);
    else
      f(p, P, col, false);
  } else {
    if (seg != 0 || tid >= 32 * NCOL) return;
    const int col = NCOL == 2 ? (tid >> 5) : col0;
    const int j = 32 * (jy - g.n[1]) + (tid & 31);
    if (j >= g.n[1]) return;
    const int q = (j + k + col) & 1;
    const int ih = q ? hn - 1 : 0;
    const int p[3] = {2 * ih + q, j, k};
    f(p, (j + g.n[1] * k) * hn + ih, col, false);
  }
}

// Position offset, within the rows of the layout, of the neighbour one step
// along axis a (s = +1 or -1) of a cell with x parity q: along x the cell
// i + 1 sits at i / 2 + q and i - 1 at i / 2 + q - 1; along y and z the rows
// are n0 / 2 (sy) and n1 n0 / 2 (sz) apart.  Offsets add for diagonal steps.
__host__ __device__ __forceinline__ int split_step(int a, int s, int q, int sy, int sz) {
  return a == 0 ? (s > 0 ? q : q - 1) : (a == 1 ? s * sy : s * sz);
}

// The values visc_gs_interior and tensor_interior gather for component c of
// an interior cell at position P of colour col (x parity q): the cell
// viscosity sums elo / ehi (CellEta's), u_c at the six face neighbours (the
// other colour), and for a != c the six values of u_a of the cross term (the
// two face neighbours along c in the other colour, the four diagonal ones in
// the cell's own colour).
struct SplitCell {
  int P, q, own, oth, sy, sz;
  __host__ __device__ __forceinline__ SplitCell(const Geom& g, int col, int q_, int P_)
      : P(P_), q(q_), own(col * (g.ncell >> 1)), oth((1 - col) * (g.ncell >> 1)), sy(g.n[0] >> 1),
        sz((g.n[0] >> 1) * g.n[1]) {}
  __host__ __device__ __forceinline__ int step(int a, int s) const { return split_step(a, s, q, sy, sz); }
};

__host__ __device__ __forceinline__ void split_eta(const float* __restrict__ eta, const SplitCell& s, float* elo,
                                                   float* ehi) {
  const float e0 = eta[s.own + s.P];
  const float* eo = eta + s.oth;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    elo[a] = eo[s.P + s.step(a, -1)] + e0;
    ehi[a] = e0 + eo[s.P + s.step(a, 1)];
  }
}

__host__ __device__ __forceinline__ void split_u(const float* __restrict__ u, const Geom& g, const SplitCell& s, int c,
                                                 float* ulo, float* uhi, float (*xa)[6]) {
  const float* uo = u + (size_t)c * g.ncell + s.oth;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ulo[a] = uo[s.P + s.step(a, -1)];
    uhi[a] = uo[s.P + s.step(a, 1)];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == c) continue;
    const float* ao = u + (size_t)a * g.ncell + s.oth;
    const float* aw = u + (size_t)a * g.ncell + s.own;
    const int cp = s.step(c, 1), cm = s.step(c, -1), ap = s.step(a, 1), am = s.step(a, -1);
    xa[a][0] = ao[s.P + cp];
    xa[a][1] = ao[s.P + cm];
    xa[a][2] = aw[s.P + ap + cp];
    xa[a][3] = aw[s.P + ap + cm];
    xa[a][4] = aw[s.P + am + cp];
    xa[a][5] = aw[s.P + am + cm];
  }
}

// Positions around a wall cell p (position P of colour col) in the split
// layout, for the gather forms of the wall-cell functions below: one offset
// per access instead of a full index (cells p + d inside the grid, d in
// {-1, 0, 1}^3), and the face viscosities as CellEta forms them (a wall face
// takes the cell's own).
struct SplitWall {
  int own, oth, q, P, sy, sz;
  float elo[3], ehi[3];
  __host__ __device__ __forceinline__ SplitWall(const float* __restrict__ eta, const Geom& g, int col, const int* p,
                                                int P_)
      : own(col * (g.ncell >> 1)), oth((1 - col) * (g.ncell >> 1)), q(p[0] & 1), P(P_), sy(g.n[0] >> 1),
        sz((g.n[0] >> 1) * g.n[1]) {
    const float e0 = eta[own + P];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int dm[3] = {0, 0, 0}, dp[3] = {0, 0, 0};
      dm[a] = -1;
      dp[a] = 1;
      const float em = p[a] > 0 ? eta[pos(dm)] : e0;
      const float ep = p[a] < g.n[a] - 1 ? eta[pos(dp)] : e0;
      elo[a] = 0.5f * (em + e0);
      ehi[a] = 0.5f * (e0 + ep);
    }
  }
  __host__ __device__ __forceinline__ int pos(const int* d) const {
    return (((d[0] + d[1] + d[2]) & 1) ? oth : own) + P + d[1] * sy + d[2] * sz +
           (d[0] > 0 ? q : (d[0] < 0 ? q - 1 : 0));
  }
};

// mg_face_cross of component a (u_a = ua) on the face normal to a below
// (lower) or above wall cell p, derivative along c: 0 on a wall face, values
// outside the grid along c the wall ghosts 2 u_b - u
__host__ __device__ __forceinline__ float split_face_cross(const float* __restrict__ ua, const Geom& g,
                                                           const SplitWall& w, const int* p, int a, int c, bool lower,
                                                           int hom) {
  if (lower ? p[a] == 0 : p[a] == g.n[a] - 1) return 0.f;
  auto ug = [&](int da, int dc) -> float {
    int d[3] = {0, 0, 0};
    d[a] = da;
    const int qc = p[c] + dc;
    if (qc < 0 || qc >= g.n[c]) {
      const float v = ua[w.pos(d)];
      const float ub = hom ? 0.f : g.fwu[c][qc < 0 ? 0 : 1][a];
      return rn_add(rn_mul(2.f, ub), -v);
    }
    d[c] = dc;
    return ua[w.pos(d)];
  };
  const int l = lower ? -1 : 0;
  const float dL = rn_add(ug(l, 1), -ug(l, -1));
  const float dR = rn_add(ug(l + 1, 1), -ug(l + 1, -1));
  return rn_mul(rn_add(dL, dR), g.fq4);
}

// The Gauss-Seidel value of component C at wall cell p: visc_gs_point's
// arithmetic (the same operations in the same order, so the same bits) on
// the values gathered through SplitWall.
template <int C>
__host__ __device__ __forceinline__ float split_gs_wall(const float* __restrict__ u, const float* __restrict__ b,
                                                        const float* __restrict__ eta, const Geom& g, int col,
                                                        const int* p, int P, float beta, int hom) {
  const SplitWall w(eta, g, col, p, P);
  const float* uC = u + (size_t)C * g.ncell;
  float offd = 0.f, diag = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float kappa = a == C ? 2.f : 1.f;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const float wf = kappa * (sd ? w.ehi[a] : w.elo[a]) * g.fihh;
      if (sd ? p[a] == g.n[a] - 1 : p[a] == 0) {
        const float ub = hom ? 0.f : g.fwu[a][sd][C];
        offd = rn_fma(rn_mul(2.f, wf), ub, offd);
        diag = rn_fma(2.f, wf, diag);
      } else {
        int d[3] = {0, 0, 0};
        d[a] = sd ? 1 : -1;
        offd = rn_fma(wf, uC[w.pos(d)], offd);
        diag = rn_add(diag, wf);
      }
    }
  }
  float cross = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == C) continue;
    const float* ua = u + (size_t)a * g.ncell;
    const float fluxhi = rn_mul(w.ehi[a], split_face_cross(ua, g, w, p, a, C, false, hom));
    const float fluxlo = rn_mul(w.elo[a], split_face_cross(ua, g, w, p, a, C, true, hom));
    cross = rn_fma(rn_add(fluxhi, -fluxlo), g.fih, cross);
  }
  return rn_fma(beta, rn_add(offd, cross), b[(size_t)C * g.ncell + w.own + P]) / rn_fma(beta, diag, 1.f);
}

// (L_eta u)_c at wall cell p: mg_tensor_point's arithmetic (same operations,
// same order) on the values gathered through w; u0 = u_c at p
__host__ __device__ __forceinline__ float split_lu_wall(const float* __restrict__ u, const Geom& g,
                                                        const SplitWall& w, const int* p, int c, float u0, int hom) {
  const float* uc = u + (size_t)c * g.ncell;
  float acc = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float flux[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      // the face between L = p + (sd - 1) e_a and R = L + e_a; the one outside
      // the grid is the wall ghost 2 u_b - u0
      float uL = u0, uR = u0;
      int d[3] = {0, 0, 0};
      d[a] = sd ? 1 : -1;
      const bool wall = sd ? p[a] == g.n[a] - 1 : p[a] == 0;
      const float un = wall ? rn_add(rn_mul(2.f, hom ? 0.f : g.fwu[a][sd][c]), -u0) : uc[w.pos(d)];
      if (sd)
        uR = un;
      else
        uL = un;
      const float e = sd ? w.ehi[a] : w.elo[a];
      const float nrm = rn_mul(rn_add(uR, -uL), g.fih);
      if (a == c)
        flux[sd] = rn_mul(e, rn_mul(2.f, nrm));
      else
        flux[sd] = rn_mul(e, rn_add(nrm, split_face_cross(u + (size_t)a * g.ncell, g, w, p, a, c, sd == 0, hom)));
    }
    acc = rn_add(acc, rn_mul(rn_add(flux[1], -flux[0]), g.fih));
  }
  return acc;
}

// Gauss-Seidel update of component C at wall cell p (position P) of colour col
template <int C>
__host__ __device__ __forceinline__ void split_smooth_wall(float* __restrict__ u, const float* __restrict__ b,
                                                           const float* __restrict__ eta, const Geom& g, int col,
                                                           const int* p, int P, float beta, int hom) {
  u[(size_t)C * g.ncell + (size_t)col * (g.ncell >> 1) + P] = split_gs_wall<C>(u, b, eta, g, col, p, P, beta, hom);
}

// Thread -> cells map of the sweep: the cells of the colour at positions
// i / 2 = 2t and 2t + 1 of a row per thread t (an even first position, so that
// both can be read with one 8-byte load), in 2D blocks of bx threads along the
// row (a row segment of at most 256 threads) times R rows, R chosen so that
// bx R fills whole warps where it can (48 threads per row: 2 rows, 3 warps).
// Block (seg, jb, k) with jb < nb takes rows jb R .. jb R + R - 1 of plane k:
// every cell of the row but its x-wall cell (i = 0 or n0 - 1), interior
// unless j or k is on a wall.  The blocks (0, nb + G, k) take the x-wall cells
// of rows 32 G .. 32 G + 31, one per thread of the first warp, right after the
// plane's rows.  f(p, P, interior, a, b) for the first cell p (i / 2 = 2t) at
// position P; a and b tell which of it and the next cell (p[0] + 2, P + 1)
// belong to the thread.
struct SplitSweep {
  int bx, R, nseg, nb;
};

__host__ __device__ inline SplitSweep split_sweep(const Geom& g) {
  const int pairs = ((g.n[0] >> 1) + 1) / 2;
  SplitSweep w;
  w.bx = pairs < 256 ? pairs : 256;
  w.nseg = (pairs + w.bx - 1) / w.bx;
  int gcd = w.bx, m = 32;
  while (m) {
    const int t = gcd % m;
    gcd = m;
    m = t;
  }
  w.R = 32 / gcd;
  if (w.bx * w.R > 256) w.R = 256 / w.bx > 1 ? 256 / w.bx : 1;
  if (w.bx * w.R < 32) w.R = (32 + w.bx - 1) / w.bx;  // the x-wall blocks need a warp
  w.nb = (g.n[1] + w.R - 1) / w.R;
  return w;
}

inline dim3 split_sweep_grid(const Geom& g) {
  const SplitSweep w = split_sweep(g);
  return dim3((unsigned)w.nseg, (unsigned)(w.nb + (g.n[1] + 31) / 32), (unsigned)g.n[2]);
}
inline dim3 split_sweep_block(const Geom& g) {
  const SplitSweep w = split_sweep(g);
  return dim3((unsigned)w.bx, (unsigned)w.R, 1);
}

template <typename F>
__host__ __device__ __forceinline__ void split_pair_thread(const Geom& g, int col, const SplitSweep& w, int seg, int jb,
                                                           int k, int tx, int ty, F&& f) {
  const int hn = g.n[0] >> 1;
  if (jb < w.nb) {
    const int j = jb * w.R + ty;
    const int ih = 2 * (seg * w.bx + tx);
    if (j >= g.n[1] || ih >= hn) return;
    const int q = (j + k + col) & 1;  // x parity of the colour's cells in this row
    // the row's cells but its x-wall cell: i / 2 in [1 - q, hn - 1 - q]
    const bool a = ih >= 1 - q && ih <= hn - 1 - q, b = ih + 1 <= hn - 1 - q;
    const int p[3] = {2 * ih + q, j, k};
    const int P = (j + g.n[1] * k) * hn + ih;
    if (j > 0 && j < g.n[1] - 1 && k > 0 && k < g.n[2] - 1)
      f(p, P, true, a, b);
    else
      f(p, P, false, a, b);
  } else {
    const int t = ty * w.bx + tx;
    if (seg != 0 || t >= 32) return;
    const int j = 32 * (jb - w.nb) + t;
    if (j >= g.n[1]) return;
    const int q = (j + k + col) & 1;
    const int ih = q ? hn - 1 : 0;
    const int p[3] = {2 * ih + q, j, k};
    f(p, (j + g.n[1] * k) * hn + ih, false, true, false);
  }
}

// two floats at an even position of a (8-byte aligned)
__host__ __device__ __forceinline__ void ld2(const float* __restrict__ a, int pos, float& x0, float& x1) {
#ifdef __CUDA_ARCH__
  const float2 v = *reinterpret_cast<const float2*>(a + pos);
  x0 = v.x;
  x1 = v.y;
#else
  x0 = a[pos];
  x1 = a[pos + 1];
#endif
}

// The values two interior cells of colour col at positions P0 (even) and
// P0 + 1 (x parity q) read, by 8-byte loads: a neighbour displaced along y or
// z sits at P0 + d for the first cell and P0 + d + 1 for the second (one
// load); along x the two cells need three consecutive positions from
// P0 + q - 1 or P0 + q (one 8-byte load at the even position and one 4-byte
// load).  get(arr, a1, s1, a2, s2): the pair's values of arr (a colour's half)
// at the displacement s1 e_a1 + s2 e_a2 (a2 < 0: none).
struct SplitPair {
  int P0, q, own, oth, dr[3];
  __host__ __device__ __forceinline__ SplitPair(const Geom& g, int col, int q_, int P0_)
      : P0(P0_), q(q_), own(col * (g.ncell >> 1)), oth((1 - col) * (g.ncell >> 1)), dr{0, g.n[0] >> 1, (g.n[0] >> 1) * g.n[1]} {}
  __host__ __device__ __forceinline__ void get(const float* __restrict__ arr, int a1, int s1, int a2, int s2, float& xa,
                                               float& xb) const {
    int off = 0, sx = 0;
    if (a1 == 0)
      sx = s1;
    else
      off += s1 * dr[a1];
    if (a2 == 0)
      sx = s2;
    else if (a2 > 0)
      off += s2 * dr[a2];
    const int base = P0 + off;
    float v0, v1;
    ld2(arr, base, v0, v1);
    if (sx > 0) {  // base + q and base + q + 1
      const float s = arr[base + 2];
      xa = q ? v1 : v0;
      xb = q ? s : v1;
    } else if (sx < 0) {  // base + q - 1 and base + q
      const float s = arr[base - 1];
      xa = q ? v0 : s;
      xb = q ? v1 : v0;
    } else {
      xa = v0;
      xb = v1;
    }
  }
  // CellEta's face sums of the pair (elo / ehi as split_eta forms them)
  __host__ __device__ __forceinline__ void eta(const float* __restrict__ e, float (*elo)[3], float (*ehi)[3]) const {
    float e0a, e0b;
    ld2(e + own, P0, e0a, e0b);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float la, lb, ha, hb;
      get(e + oth, a, -1, -1, 0, la, lb);
      get(e + oth, a, 1, -1, 0, ha, hb);
      elo[0][a] = la + e0a;
      elo[1][a] = lb + e0b;
      ehi[0][a] = e0a + ha;
      ehi[1][a] = e0b + hb;
    }
  }
  // u_c at the face neighbours and, for a != c, the cross term's u_a values
  // (split_u's) of the pair
  __host__ __device__ __forceinline__ void stencil(const float* __restrict__ u, const Geom& g, int c, float (*ulo)[3],
                                                   float (*uhi)[3], float (*xa)[3][6]) const {
    const float* uo = u + (size_t)c * g.ncell + oth;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      get(uo, a, -1, -1, 0, ulo[0][a], ulo[1][a]);
      get(uo, a, 1, -1, 0, uhi[0][a], uhi[1][a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == c) continue;
      const float* ao = u + (size_t)a * g.ncell + oth;
      const float* aw = u + (size_t)a * g.ncell + own;
      get(ao, c, 1, -1, 0, xa[0][a][0], xa[1][a][0]);
      get(ao, c, -1, -1, 0, xa[0][a][1], xa[1][a][1]);
      get(aw, a, 1, c, 1, xa[0][a][2], xa[1][a][2]);
      get(aw, a, 1, c, -1, xa[0][a][3], xa[1][a][3]);
      get(aw, a, -1, c, 1, xa[0][a][4], xa[1][a][4]);
      get(aw, a, -1, c, -1, xa[0][a][5], xa[1][a][5]);
    }
  }
};

// The Gauss-Seidel values of component C at the pair (SplitPair's cells):
// the same values as split_gs_value gathers, into the same visc_gs_core, so
// the same bits
template <int C>
__host__ __device__ __forceinline__ void split_gs_pair(const float* __restrict__ u, const float* __restrict__ b,
                                                       const float* __restrict__ eta, const Geom& g, int col, int q,
                                                       int P0, float bs, float& va, float& vb) {
  const SplitPair sp(g, col, q, P0);
  float elo[2][3], ehi[2][3], ulo[2][3], uhi[2][3], xa[2][3][6];
  sp.eta(eta, elo, ehi);
  sp.stencil(u, g, C, ulo, uhi, xa);
  float ba, bb;
  ld2(b + (size_t)C * g.ncell + sp.own, P0, ba, bb);
  va = visc_gs_core<3, float>(C, elo[0], ehi[0], ulo[0], uhi[0], xa[0], ba, bs);
  vb = visc_gs_core<3, float>(C, elo[1], ehi[1], ulo[1], uhi[1], xa[1], bb, bs);
}

// the Gauss-Seidel value of component C at interior cell s
template <int C>
__host__ __device__ __forceinline__ float split_gs_value(const float* __restrict__ u, const float* __restrict__ b,
                                                         const float* __restrict__ eta, const Geom& g,
                                                         const SplitCell& s, float bs) {
  float elo[3], ehi[3], ulo[3], uhi[3], xa[3][6];
  split_eta(eta, s, elo, ehi);
  split_u(u, g, s, C, ulo, uhi, xa);
  return visc_gs_core<3, float>(C, elo, ehi, ulo, uhi, xa, b[(size_t)C * g.ncell + s.own + s.P], bs);
}

// thread (tx, ty) of block (seg, jb, k) of a sweep of colour col: both values
// of an interior pair are formed before either is stored, so that the loads
// the two cells share are issued once (the stores, to u_C of colour col, hit
// no value either cell reads).  VEC: the pair read by 8-byte loads
// (split_gs_pair; n0 / 2 even and 8-byte aligned arrays).
template <int C, bool VEC>
__host__ __device__ __forceinline__ void split_smooth_thread(float* __restrict__ u, const float* __restrict__ b,
                                                             const float* __restrict__ eta, const Geom& g, int col,
                                                             float beta, int hom, const SplitSweep& w, int seg, int jb,
                                                             int k, int tx, int ty) {
  const float bs = beta * (g.fihh * 0.5f);  // CellEta's factor 1/2 with 1/h^2
  split_pair_thread(g, col, w, seg, jb, k, tx, ty, [&](const int* p, int P, bool in, bool ca, bool cb) {
    const size_t o = (size_t)C * g.ncell + (size_t)col * (g.ncell >> 1) + P;
    if (in) {
      float va, vb;
      if (VEC) {
        split_gs_pair<C>(u, b, eta, g, col, p[0] & 1, P, bs, va, vb);
      } else {
        if (ca) va = split_gs_value<C>(u, b, eta, g, SplitCell(g, col, p[0] & 1, P), bs);
        if (cb) vb = split_gs_value<C>(u, b, eta, g, SplitCell(g, col, p[0] & 1, P + 1), bs);
      }
#ifdef __CUDA_ARCH__
      if (VEC && ca && cb) {
        *reinterpret_cast<float2*>(u + o) = make_float2(va, vb);
        return;
      }
#endif
      if (ca) u[o] = va;
      if (cb) u[o + 1] = vb;
    } else {
      if (ca) split_smooth_wall<C>(u, b, eta, g, col, p, P, beta, hom);
      if (cb) {
        const int p2[3] = {p[0] + 2, p[1], p[2]};
        split_smooth_wall<C>(u, b, eta, g, col, p2, P + 1, beta, hom);
      }
    }
  });
}

// Red-black Gauss-Seidel sweep of component C over the cells of colour col
// (the update of k_visc_smooth_c with the cell viscosity); grid
// split_sweep_grid(g), block split_sweep_block(g).  VEC: see
// split_smooth_thread; it holds both cells' values at once and runs at 64
// registers (at 40 or 48 it spilled and was slower than the scalar form; at
// 64, 72-76 against 75-82 us per 256^3 launch).
template <int C, bool VEC>
__global__ void __launch_bounds__(256, VEC ? 4 : 6) k_visc_smooth_split(float* __restrict__ u, const float* __restrict__ b,
                                                               const float* __restrict__ eta,
                                                               const __grid_constant__ Geom g, int col, float beta,
                                                               int hom) {
  // the map's sizes are the launch's (split_sweep(g) on the host)
  const SplitSweep w{(int)blockDim.x, (int)blockDim.y, (int)gridDim.x, (int)gridDim.y - (g.n[1] + 31) / 32};
  split_smooth_thread<C, VEC>(u, b, eta, g, col, beta, hom, w, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x,
                              threadIdx.y);
}

// the operator at a wall cell
__host__ __device__ __forceinline__ void split_op_wall(const float* __restrict__ u, const float* __restrict__ b,
                                                    float* __restrict__ out, const float* __restrict__ eta,
                                                    const Geom& g, float beta, int hom, int col, const int* p, int P) {
  const SplitWall w(eta, g, col, p, P);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t o = (size_t)c * g.ncell + w.own + P;
    const float Lu = split_lu_wall(u, g, w, p, c, u[o], hom);
    out[o] = op_out<float>(u[o], Lu, beta, b, o);
  }
}

// out = u - beta L u, or r = b - (u - beta L u) when b != nullptr, for every
// component of cell p (position P) of colour col: the operator of k_visc_op3
// with the cell viscosity
template <bool IN>
__host__ __device__ __forceinline__ void split_op_cell(const float* __restrict__ u, const float* __restrict__ b,
                                                       float* __restrict__ out, const float* __restrict__ eta,
                                                       const Geom& g, float beta, int hom, int col, const int* p,
                                                       int P) {
  if (IN) {
    const SplitCell s(g, col, p[0] & 1, P);
    const float sc = g.fihh * 0.5f;
    float elo[3], ehi[3];
    split_eta(eta, s, elo, ehi);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float ulo[3], uhi[3], xa[3][6];
      split_u(u, g, s, c, ulo, uhi, xa);
      const size_t o = (size_t)c * g.ncell + s.own + P;
      const float Lu = tensor_core<3, float>(c, u[o], elo, ehi, ulo, uhi, xa, sc);
      out[o] = op_out<float>(u[o], Lu, beta, b, o);
    }
  } else {
    split_op_wall(u, b, out, eta, g, beta, hom, col, p, P);
  }
}

// thread tid of block (seg, j, k) of the operator (both colours of the row)
__host__ __device__ __forceinline__ void split_op_thread(const float* __restrict__ u, const float* __restrict__ b,
                                                         float* __restrict__ out, const float* __restrict__ eta,
                                                         const Geom& g, float beta, int hom, int seg, int j, int k,
                                                         int tid) {
  const SplitMap sm = split_map(g);
  split_thread<2>(g, 0, sm.W, seg, j, k, tid, [&](const int* p, int P, int col, bool in) {
    if (in)
      split_op_cell<true>(u, b, out, eta, g, beta, hom, col, p, P);
    else
      split_op_cell<false>(u, b, out, eta, g, beta, hom, col, p, P);
  });
}

// grid split_grid(g), block split_block_dim(g, 2)
__global__ void __maxnreg__(64) k_visc_op_split(const float* __restrict__ u,
                                                                        const float* __restrict__ b,
                                                                        float* __restrict__ out,
                                                                        const float* __restrict__ eta,
                                                                        const __grid_constant__ Geom g, float beta,
                                                                        int hom) {
  split_op_thread(u, b, out, eta, g, beta, hom, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x);
}

// Pair s (0 <= s < ncell / 2) of neighbouring cells (2 ih, 2 ih + 1) of a row:
// natural index of the first and colour of the first; both sit at position
// s of their colour's half.
__host__ __device__ __forceinline__ void split_pair(const Geom& g, int s, size_t& nat, int& c0) {
  const int hn = g.n[0] >> 1;
  const int row = divm(s, hn, g.m_rb);
  const int ih = s - row * hn;
  const int k = divm(row, g.n[1], g.m_n1);
  const int j = row - k * g.n[1];
  nat = (size_t)row * g.n[0] + 2 * ih;
  c0 = (j + k) & 1;
}

// pair tt of ncomp components: out (split, FP32) = a - bsub (natural, FP64;
// a alone when bsub is null), the conversions of k_convert and k_diff_to_f32
__host__ __device__ __forceinline__ void split_from_pair(float* __restrict__ out, const double* __restrict__ a,
                                                         const double* __restrict__ bsub, const Geom& g,
                                                         long long tt) {
  const int half = g.ncell >> 1;
  const int comp = tt >= half ? (tt >= 2LL * half ? 2 : 1) : 0;
  const int s = (int)(tt - (long long)comp * half);
  size_t nat;
  int c0;
  split_pair(g, s, nat, c0);
  const size_t base = (size_t)comp * g.ncell;
  const float v0 = bsub ? (float)(a[base + nat] - bsub[base + nat]) : (float)a[base + nat];
  const float v1 = bsub ? (float)(a[base + nat + 1] - bsub[base + nat + 1]) : (float)a[base + nat + 1];
  out[base + (size_t)c0 * half + s] = v0;
  out[base + (size_t)(1 - c0) * half + s] = v1;
}

// pair tt: x (natural, FP64) += sc d (split, FP32), the updates of k_add_f32
// and k_add_scaled_f32
__host__ __device__ __forceinline__ void split_add_pair(double* __restrict__ x, double sc, const float* __restrict__ d,
                                                        const Geom& g, long long tt) {
  const int half = g.ncell >> 1;
  const int comp = tt >= half ? (tt >= 2LL * half ? 2 : 1) : 0;
  const int s = (int)(tt - (long long)comp * half);
  size_t nat;
  int c0;
  split_pair(g, s, nat, c0);
  const size_t base = (size_t)comp * g.ncell;
  x[base + nat] += sc * (double)d[base + (size_t)c0 * half + s];
  x[base + nat + 1] += sc * (double)d[base + (size_t)(1 - c0) * half + s];
}

// grid-stride over the ncomp ncell / 2 pairs
__global__ void k_split_from(float* __restrict__ out, const double* __restrict__ a, const double* __restrict__ bsub,
                             const __grid_constant__ Geom g, int ncomp) {
  const long long tot = (long long)ncomp * (g.ncell >> 1);
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < tot;
       tt += (long long)gridDim.x * blockDim.x)
    split_from_pair(out, a, bsub, g, tt);
}

__global__ void k_split_add(double* __restrict__ x, double sc, const float* __restrict__ d,
                            const __grid_constant__ Geom g, int ncomp) {
  const long long tot = (long long)ncomp * (g.ncell >> 1);
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < tot;
       tt += (long long)gridDim.x * blockDim.x)
    split_add_pair(x, sc, d, g, tt);
}

}  // namespace hb
