// Multigrid kernels for the three solves of the step, templated on the space
// dimension D and the arithmetic type T (double for the FP64 path, float for
// the FP32 V-cycles of the mixed-precision defect correction).
//
//  * tensor viscous: (I - beta L_eta) u = b, red-black Gauss-Seidel on one
//    component at a time with the other components frozen in the cross terms
//  * cell Poisson (MAC potential): red-black Gauss-Seidel, Neumann walls
//  * nodal FE Poisson: 2^D-colour Gauss-Seidel (the 3^D stencil couples
//    diagonal neighbours), Neumann walls by even reflection
//  * transfers: cell averaging / cell-centred multilinear interpolation,
//    full weighting / multilinear interpolation on nodes, coarse face eta as
//    the mean of the fine faces tiling each coarse face
#pragma once
#include <cmath>
#include "hb_common.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// tensor viscous operator pieces (mirrors the explicit-stage operator)
// ---------------------------------------------------------------------------
// Explicitly rounded FP32 operations (round to nearest): the compiler may not
// contract or reorder them, so every kernel that inlines the Gauss-Seidel
// point updates and the operator core below (visc_gs_point, visc_gs_core,
// tensor_core) issues the same FP32 operations in the same order and gets the
// same bits (the staged and unstaged FP32 kernels are checked against each
// other bit for bit).  The FP64 forms are the plain operations, which the
// compiler may fuse: the FP64 kernels are bound by GB300's FP64 issue rate,
// and none of them has a second implementation to agree with.  On the host
// (the host-built checks) both are the plain operations and an exact fused
// multiply-add.
template <typename T>
__host__ __device__ __forceinline__ T rn_mul(T a, T b);
template <typename T>
__host__ __device__ __forceinline__ T rn_add(T a, T b);
template <typename T>
__host__ __device__ __forceinline__ T rn_fma(T a, T b, T c);
template <>
__host__ __device__ __forceinline__ float rn_mul<float>(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
template <>
__host__ __device__ __forceinline__ double rn_mul<double>(double a, double b) {
  return a * b;
}
template <>
__host__ __device__ __forceinline__ float rn_add<float>(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
template <>
__host__ __device__ __forceinline__ double rn_add<double>(double a, double b) {
  return a + b;
}
template <>
__host__ __device__ __forceinline__ float rn_fma<float>(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
template <>
__host__ __device__ __forceinline__ double rn_fma<double>(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return a * b + c;
#else
  return std::fma(a, b, c);
#endif
}

struct Strides;

// The face viscosities of a level, stored per face (FaceEta), or, on the
// finest level of the FP32 V-cycles, formed where they are used as the mean
// of the two cells' viscosities (CellEta: the rule that makes the stored
// finest-level faces, wall faces taking the interior cell; one cell array is
// read instead of D face arrays).
//   lo / hi: the face of axis a below / above interior cell p (flat index id),
//            up to the factor kScale (CellEta returns the two cells' sum)
//   at:      the face of axis a whose upper cell is q (q[a] may be n[a])
template <typename T>
struct FaceEta {
  static constexpr double kScale = 1.0;
  const T* const* ef;
  __host__ __device__ T lo(const Geom& g, const Strides& S, int a, const int* p, int id) const;
  __host__ __device__ T hi(const Geom& g, const Strides& S, int a, const int* p, int id) const;
  template <bool PER = true>
  __host__ __device__ T at(const Geom& g, int a, const int* q) const {
    return ef[a][fidx(g, a, q[0], q[1], q[2])];
  }
};

template <typename T>
struct CellEta {
  static constexpr double kScale = 0.5;
  const T* eta;
  __host__ __device__ T lo(const Geom& g, const Strides& S, int a, const int* p, int id) const;
  __host__ __device__ T hi(const Geom& g, const Strides& S, int a, const int* p, int id) const;
  template <bool PER = true>
  __host__ __device__ T at(const Geom& g, int a, const int* q) const {
    int L[3] = {q[0], q[1], q[2]}, R[3] = {q[0], q[1], q[2]};
    if (PER && g.per[a]) {  // periodic: the two cells across the face, wrapped
      L[a] = wrap_cell(q[a] - 1, g.n[a]);
      R[a] = wrap_cell(q[a], g.n[a]);
    } else {
      L[a] = q[a] > 0 ? q[a] - 1 : 0;
      R[a] = q[a] < g.n[a] ? q[a] : g.n[a] - 1;
    }
    return T(0.5) * (eta[cidx<3>(g, L[0], L[1], L[2])] + eta[cidx<3>(g, R[0], R[1], R[2])]);
  }
};

// component comp at cell q, which lies inside the domain on every axis but
// ax: uget with the one reflection test that can apply
template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ T uget_axis(const T* __restrict__ uc, const Geom& g, int comp, int i, int j, int k,
                                                int ax, bool hom) {
  int q[3] = {i, j, k};
  if (PER && g.per[ax]) {
    q[ax] = wrap_cell(q[ax], g.n[ax]);
    return uc[cidx<D>(g, q[0], q[1], q[2])];
  }
  int side = -1;
  if (q[ax] < 0) {
    side = 0;
    q[ax] = -q[ax] - 1;
  } else if (q[ax] >= g.n[ax]) {
    side = 1;
    q[ax] = 2 * g.n[ax] - 1 - q[ax];
  }
  const T v = uc[cidx<D>(g, q[0], q[1], q[2])];
  if (side < 0) return v;
  const T ub = hom ? T(0) : g_wu<T>(g, ax, side, comp);
  return rn_add(rn_mul(T(2), ub), -v);
}

template <int D, typename T, bool PER = true>
__host__ __device__ inline T mg_face_cross(const T* __restrict__ ua, const Geom& g, int a, int c, const int* L,
                                  bool hom) {
  // mean of the two cells' central differences, (dL + dR)/2 with dL, dR over 2h;
  // on a wall axis L and L + e_a are inside the domain (a wall face gives 0),
  // on a periodic axis they are wrapped, so only the c offsets can leave it
  const bool pa = PER && g.per[a];
  if (!pa && (L[a] < 0 || L[a] >= g.n[a] - 1)) return T(0);
  int p1[3] = {L[0], L[1], L[2]}, p0[3] = {L[0], L[1], L[2]};
  if (pa) p1[a] = p0[a] = wrap_cell(L[a], g.n[a]);
  p1[c] += 1;
  p0[c] -= 1;
  T dL = rn_add(uget_axis<D, T, PER>(ua, g, a, p1[0], p1[1], p1[2], c, hom),
                -uget_axis<D, T, PER>(ua, g, a, p0[0], p0[1], p0[2], c, hom));
  if (pa) {
    p1[a] = p0[a] = wrap_cell(L[a] + 1, g.n[a]);
  } else {
    p1[a] += 1;
    p0[a] += 1;
  }
  T dR = rn_add(uget_axis<D, T, PER>(ua, g, a, p1[0], p1[1], p1[2], c, hom),
                -uget_axis<D, T, PER>(ua, g, a, p0[0], p0[1], p0[2], c, hom));
  return rn_mul(rn_add(dL, dR), g_q4<T>(g));
}

template <int D, typename T, bool PER = true, typename EF>
__host__ __device__ inline T mg_tensor_point(const T* __restrict__ u, const EF& ef, const Geom& g, int c,
                                    const int* p, bool hom) {
  const T* uc = u + (size_t)c * g.ncell;
  T acc = T(0);
  const T ih = g_ih<T>(g);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T flux[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      int L[3] = {p[0], p[1], p[2]};
      L[a] += s - 1;
      int R[3] = {L[0], L[1], L[2]};
      R[a] += 1;
      T e = ef.template at<PER>(g, a, R);
      // L and R differ from the cell p only along a
      T nrm = rn_mul(rn_add(uget_axis<D, T, PER>(uc, g, c, R[0], R[1], R[2], a, hom),
                            -uget_axis<D, T, PER>(uc, g, c, L[0], L[1], L[2], a, hom)),
                     ih);
      if (a == c)
        flux[s] = rn_mul(e, rn_mul(T(2), nrm));
      else
        flux[s] = rn_mul(e, rn_add(nrm, mg_face_cross<D, T, PER>(u + (size_t)a * g.ncell, g, a, c, L, hom)));
    }
    acc = rn_add(acc, rn_mul(rn_add(flux[1], -flux[0]), ih));
  }
  return acc;
}

// Gauss-Seidel update of component c at cell p (all other values frozen)
template <int D, typename T, bool PER = true, typename EF>
__host__ __device__ inline T visc_gs_point(const T* __restrict__ u, const T* __restrict__ b, const EF& ef,
                                  const Geom& g, int c, const int* p, T beta, bool hom) {
  const T* uc = u + (size_t)c * g.ncell;
  const T ih = g_ih<T>(g);
  const T ihh = g_ihh<T>(g);
  T offd = T(0), diag = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T kappa = (a == c) ? T(2) : T(1);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      int q[3] = {p[0], p[1], p[2]};
      int fq[3] = {p[0], p[1], p[2]};
      if (s == 0) {
        q[a] -= 1;
      } else {
        q[a] += 1;
        fq[a] += 1;
      }
      T wf = kappa * ef.template at<PER>(g, a, fq) * ihh;
      const bool pa = PER && g.per[a];
      bool wall = !pa && ((s == 0) ? (p[a] == 0) : (p[a] == g.n[a] - 1));
      if (wall) {
        T ub = hom ? T(0) : g_wu<T>(g, a, s, c);
        offd = rn_fma(rn_mul(T(2), wf), ub, offd);
        diag = rn_fma(T(2), wf, diag);
      } else {
        if (pa) q[a] = wrap_cell(q[a], g.n[a]);
        offd = rn_fma(wf, uc[cidx<D>(g, q[0], q[1], q[2])], offd);
        diag = rn_add(diag, wf);
      }
    }
  }
  T cross = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == c) continue;
    const T* ua = u + (size_t)a * g.ncell;
    int Llo[3] = {p[0], p[1], p[2]};
    Llo[a] -= 1;
    int fhi[3] = {p[0], p[1], p[2]};
    fhi[a] += 1;
    T fluxhi = rn_mul(ef.template at<PER>(g, a, fhi), mg_face_cross<D, T, PER>(ua, g, a, c, p, hom));
    T fluxlo = rn_mul(ef.template at<PER>(g, a, p), mg_face_cross<D, T, PER>(ua, g, a, c, Llo, hom));
    cross = rn_fma(rn_add(fluxhi, -fluxlo), ih, cross);
  }
  // explicitly rounded (see rn_fma): the same result wherever it is inlined
  return rn_fma(beta, rn_add(offd, cross), b[(size_t)c * g.ncell + cidx<D>(g, p[0], p[1], p[2])]) /
         rn_fma(beta, diag, T(1));
}

// Strides of the cell array and of the face arrays (face array a, axis b).
struct Strides {
  int s[3];
  int fs[3][3];
};

__host__ __device__ inline Strides make_strides(const Geom& g) {
  Strides st;
  st.s[0] = 1;
  st.s[1] = g.n[0];
  st.s[2] = g.n[0] * g.n[1];
  for (int a = 0; a < 3; ++a) {
    int ex = g.n[0] + (a == 0), ey = g.n[1] + (a == 1);
    st.fs[a][0] = 1;
    st.fs[a][1] = ex;
    st.fs[a][2] = ex * ey;
  }
  return st;
}

template <typename T>
__host__ __device__ __forceinline__ T FaceEta<T>::lo(const Geom& g, const Strides& S, int a, const int* p, int id) const {
  (void)S;
  (void)id;
  return ef[a][fidx(g, a, p[0], p[1], p[2])];
}
template <typename T>
__host__ __device__ __forceinline__ T FaceEta<T>::hi(const Geom& g, const Strides& S, int a, const int* p, int id) const {
  (void)id;
  return ef[a][fidx(g, a, p[0], p[1], p[2]) + S.fs[a][a]];
}
template <typename T>
__host__ __device__ __forceinline__ T CellEta<T>::lo(const Geom& g, const Strides& S, int a, const int* p, int id) const {
  (void)g;
  (void)p;
  return eta[id - S.s[a]] + eta[id];
}
template <typename T>
__host__ __device__ __forceinline__ T CellEta<T>::hi(const Geom& g, const Strides& S, int a, const int* p, int id) const {
  (void)g;
  (void)p;
  return eta[id] + eta[id + S.s[a]];
}

template <int D>
__host__ __device__ inline bool interior(const Geom& g, const int* p) {
  bool in = p[0] >= 1 && p[0] <= g.n[0] - 2 && p[1] >= 1 && p[1] <= g.n[1] - 2;
  if (D == 3) in = in && p[2] >= 1 && p[2] <= g.n[2] - 2;
  return in;
}

// The arithmetic of the interior Gauss-Seidel update of component c on
// gathered values: elo / ehi the face viscosities below / above the cell on
// each axis (up to the accessor's factor, which is folded into bs with
// beta / h^2), ulo / uhi u_c at the two face neighbours on each axis, bc the
// right-hand side, and for each axis a != c the six values of u_a that the
// cross term reads, xa[a] = {u_a(p + e_c), u_a(p - e_c), u_a(p + e_a + e_c),
// u_a(p + e_a - e_c), u_a(p - e_a + e_c), u_a(p - e_a - e_c)}.  The update is
//   (bc + bs (offd + cross / 4)) / (1 + bs diag),
//   offd = sum_a k_a (elo_a u_lo,a + ehi_a u_hi,a), diag = sum_a k_a (elo_a + ehi_a),
//   cross = sum_{a != c} (ehi_a xhi_a - elo_a xlo_a), k_c = 2, k_a = 1 otherwise,
// in explicitly rounded operations: every caller that gathers the same
// values gets the same result bit for bit.
template <int D, typename T>
__host__ __device__ __forceinline__ T visc_gs_core(int c, const T* elo, const T* ehi, const T* ulo, const T* uhi,
                                                   const T (*xa)[6], T bc, T bs) {
  T offd = T(0), diag = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T f = rn_fma(elo[a], ulo[a], rn_mul(ehi[a], uhi[a]));
    const T w = rn_add(elo[a], ehi[a]);
    offd = a == c ? rn_fma(T(2), f, offd) : rn_add(offd, f);
    diag = a == c ? rn_fma(T(2), w, diag) : rn_add(diag, w);
  }
  T cross = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == c) continue;
    const T mid = rn_add(xa[a][0], -xa[a][1]);
    const T xhi = rn_add(mid, rn_add(xa[a][2], -xa[a][3]));
    const T xlo = rn_add(rn_add(xa[a][4], -xa[a][5]), mid);
    cross = rn_add(cross, rn_fma(ehi[a], xhi, -rn_mul(elo[a], xlo)));
  }
  const T num = rn_fma(bs, rn_fma(T(0.25), cross, offd), bc);
  const T den = rn_fma(bs, diag, T(1));
  return num / den;
}

// The same Gauss-Seidel update as visc_gs_point for a cell whose whole
// stencil is inside the domain: direct strided indexing, no ghost logic.
template <int D, typename T, typename EF>
__host__ __device__ __forceinline__ T visc_gs_interior(const T* __restrict__ u, const T* __restrict__ b, const EF& ef,
                                              const Geom& g, const Strides& S, int c, const int* p, T beta) {
  // every term of the update is linear in the face viscosities: they enter
  // unscaled, and 1/h^2 with the accessor's factor goes into beta
  const int id = cidx<D>(g, p[0], p[1], p[2]);
  const T* uc = u + (size_t)c * g.ncell;
  const T bs = beta * (g_ihh<T>(g) * T(EF::kScale));
  T elo[3], ehi[3], ulo[3], uhi[3], xa[3][6];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    elo[a] = ef.lo(g, S, a, p, id);
    ehi[a] = ef.hi(g, S, a, p, id);
    ulo[a] = uc[id - S.s[a]];
    uhi[a] = uc[id + S.s[a]];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == c) continue;
    const T* ua = u + (size_t)a * g.ncell;
    const int sa = S.s[a], sc = S.s[c];
    xa[a][0] = ua[id + sc];
    xa[a][1] = ua[id - sc];
    xa[a][2] = ua[id + sa + sc];
    xa[a][3] = ua[id + sa - sc];
    xa[a][4] = ua[id - sa + sc];
    xa[a][5] = ua[id - sa - sc];
  }
  return visc_gs_core<D, T>(c, elo, ehi, ulo, uhi, xa, b[(size_t)c * g.ncell + id], bs);
}

// (L_eta u)_c of an interior cell on gathered values (the names of
// visc_gs_core; u0 = u_c at the cell): the operator of mg_tensor_point with
// the 1/h of the differences and of the divergence taken out as one factor
// 1/h^2 (fewer multiplications; the FP64 residuals are bound by GB300's FP64
// rate), scaled by sc = 1/h^2 times the accessor's factor.  Explicitly
// rounded, like visc_gs_core: every caller that gathers the same values gets
// the same bits.
template <int D, typename T>
__host__ __device__ __forceinline__ T tensor_core(int c, T u0, const T* elo, const T* ehi, const T* ulo, const T* uhi,
                                                  const T (*xa)[6], T sc) {
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T dlo = rn_add(u0, -ulo[a]);
    const T dhi = rn_add(uhi[a], -u0);
    T flo, fhi;
    if (a == c) {
      flo = rn_mul(elo[a], rn_mul(T(2), dlo));
      fhi = rn_mul(ehi[a], rn_mul(T(2), dhi));
    } else {
      const T mid = rn_add(xa[a][0], -xa[a][1]);
      const T xhi = rn_add(mid, rn_add(xa[a][2], -xa[a][3]));
      const T xlo = rn_add(rn_add(xa[a][4], -xa[a][5]), mid);
      flo = rn_mul(elo[a], rn_fma(T(0.25), xlo, dlo));
      fhi = rn_mul(ehi[a], rn_fma(T(0.25), xhi, dhi));
    }
    acc = rn_add(acc, rn_add(fhi, -flo));
  }
  return rn_mul(acc, sc);
}

// (L_eta u)_c for an interior cell: direct strided indexing, no ghost logic
template <int D, typename T, typename EF>
__host__ __device__ __forceinline__ T tensor_interior(const T* __restrict__ u, const EF& ef, const Geom& g,
                                             const Strides& S, int c, const int* p) {
  const int id = cidx<D>(g, p[0], p[1], p[2]);
  const T* uc = u + (size_t)c * g.ncell;
  T elo[3], ehi[3], ulo[3], uhi[3], xa[3][6];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    elo[a] = ef.lo(g, S, a, p, id);
    ehi[a] = ef.hi(g, S, a, p, id);
    ulo[a] = uc[id - S.s[a]];
    uhi[a] = uc[id + S.s[a]];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == c) continue;
    const T* ua = u + (size_t)a * g.ncell;
    const int sa = S.s[a], sc = S.s[c];
    xa[a][0] = ua[id + sc];
    xa[a][1] = ua[id - sc];
    xa[a][2] = ua[id + sa + sc];
    xa[a][3] = ua[id + sa - sc];
    xa[a][4] = ua[id - sa + sc];
    xa[a][5] = ua[id - sa - sc];
  }
  return tensor_core<D, T>(c, uc[id], elo, ehi, ulo, uhi, xa, g_ihh<T>(g) * T(EF::kScale));
}

// the operator's output from (L_eta u)_c: u - beta L u, or b - (u - beta L u)
template <typename T>
__host__ __device__ __forceinline__ T op_out(T u0, T Lu, T beta, const T* b, size_t o) {
  const T Au = rn_fma(-beta, Lu, u0);
  return b ? rn_add(b[o], -Au) : Au;
}

// thread t -> cell of red-black colour col (x index stride 2)
template <int D>
__host__ __device__ inline bool rb_cell(const Geom& g, int t, int col, int* p) {
  const int nxh = (g.n[0] + 1) / 2;
  const int r = divm(t, nxh, g.m_rb);
  const int ih = t - r * nxh;
  int j, k;
  if (D == 3) {
    k = divm(r, g.n[1], g.m_n1);
    j = r - k * g.n[1];
  } else {
    j = r;
    k = 0;
  }
  int i = 2 * ih + ((j + k + col) & 1);
  p[0] = i;
  p[1] = j;
  p[2] = k;
  return i < g.n[0];
}

template <int D>
__host__ __device__ inline int rb_count(const Geom& g) {
  return ((g.n[0] + 1) / 2) * g.n[1] * (D == 3 ? g.n[2] : 1);
}

// Gauss-Seidel update of component C at cell p of the current colour
template <int D, typename T, int C, bool PER = true, typename EF>
__host__ __device__ __forceinline__ void visc_smooth_cell(T* __restrict__ u, const T* __restrict__ b, const EF& ef,
                                                          const Geom& g, T beta, int hom, const int* p) {
  T v;
  if (interior<D>(g, p)) {
    const Strides S = make_strides(g);
    v = visc_gs_interior<D, T>(u, b, ef, g, S, C, p, beta);
  } else {
    v = visc_gs_point<D, T, PER>(u, b, ef, g, C, p, beta, hom != 0);
  }
  u[(size_t)C * g.ncell + cidx<D>(g, p[0], p[1], p[2])] = v;
}

template <int D, typename T, int C, bool PER = true>
__host__ __device__ __forceinline__ void k_visc_smooth_c_at(T* __restrict__ u, const T* __restrict__ b, const T* ef0,
                                                           const T* ef1, const T* ef2, const Geom& g, int col, T beta,
                                                           int hom, int t) {
  int p[3];
  if (!rb_cell<D>(g, t, col, p)) return;
  const T* ef[3] = {ef0, ef1, ef2};
  visc_smooth_cell<D, T, C, PER>(u, b, FaceEta<T>{ef}, g, beta, hom, p);
}

// Thread -> cell maps that keep the x-wall cells out of the warps of x-interior
// cells.  A warp holding one wall cell issues the wall stencil (ghost values,
// many branches) on top of the interior one; in a row-major map a quarter of
// the warps along a 256-cell row hold one.  Rows are taken in groups of
// kMapRows: the x-interior slots (1 <= i <= n0 - 2) of the group's rows, M per
// row, then the group's 2 kMapRows wall slots (one warp's worth), so that a
// wall cell is visited soon after the interior cells of its row, while their
// cache lines are still in L2.  Rows with j or k on a wall are whole warps of
// wall cells.  (The multipliers of M and of the group size 16 M + 32 are in
// Geom; kMapRows is fixed at 16 to match.)
constexpr int kMapRows = 16;

template <int D>
__host__ __device__ inline int map_rows(const Geom& g) {
  return g.n[1] * (D == 3 ? g.n[2] : 1);
}

template <int D>
__host__ __device__ inline void row_jk(const Geom& g, int r, int* p) {
  if (D == 3) {
    p[2] = divm(r, g.n[1], g.m_n1);
    p[1] = r - p[2] * g.n[1];
  } else {
    p[1] = r;
    p[2] = 0;
  }
}

template <int D>
__host__ __device__ inline int grouped_count(const Geom& g, int M) {
  return (map_rows<D>(g) + kMapRows - 1) / kMapRows * (kMapRows * M + 2 * kMapRows);
}

// slot t -> row and m: an interior slot 0 <= m < M, or the wall slot of side
// -1 - m (x = 0 for m = -1, x = n0 - 1 for m = -2); false past the last row
template <int D>
__host__ __device__ inline bool grouped_slot(const Geom& g, int t, int M, unsigned long long mS,
                                             unsigned long long mM, int& row, int& m) {
  const int S = kMapRows * M + 2 * kMapRows;
  const int grp = divm(t, S, mS);
  int rem = t - grp * S;
  if (rem < kMapRows * M) {
    const int r = divm(rem, M, mM);
    row = grp * kMapRows + r;
    m = rem - r * M;
  } else {
    rem -= kMapRows * M;
    row = grp * kMapRows + (rem >> 1);
    m = -1 - (rem & 1);
  }
  return row < map_rows<D>(g);
}

// every cell: M = n0 - 2 interior slots per row (i = 1 + m)
template <int D>
__host__ __device__ inline int xi_count(const Geom& g) {
  return grouped_count<D>(g, g.n[0] > 2 ? g.n[0] - 2 : 0);
}

template <int D>
__host__ __device__ inline bool xi_cell(const Geom& g, int t, int* p) {
  int row, m;
  if (!grouped_slot<D>(g, t, g.n[0] > 2 ? g.n[0] - 2 : 0, g.m_xig, g.m_xi, row, m)) return false;
  row_jk<D>(g, row, p);
  if (m >= 0) {
    p[0] = 1 + m;
    return true;
  }
  p[0] = m == -1 ? 0 : g.n[0] - 1;
  return !(m == -2 && g.n[0] < 2);
}

// the cells of red-black colour col: M = (n0 - 1) / 2 interior slots per row
// (i = 2 + 2m - q with q = (j + k + col) & 1, so that i + j + k + col is
// even), and the wall slots, each taken when its cell has the colour
template <int D>
__host__ __device__ inline int rbx_count(const Geom& g) {
  return grouped_count<D>(g, (g.n[0] - 1) / 2);
}

template <int D>
__host__ __device__ inline bool rbx_cell(const Geom& g, int t, int col, int* p) {
  int row, m;
  if (!grouped_slot<D>(g, t, (g.n[0] - 1) / 2, g.m_rbxg, g.m_rbx, row, m)) return false;
  row_jk<D>(g, row, p);
  if (m >= 0) {
    p[0] = 2 + 2 * m - ((p[1] + p[2] + col) & 1);
    return p[0] <= g.n[0] - 2;
  }
  p[0] = m == -1 ? 0 : g.n[0] - 1;
  if (m == -2 && g.n[0] < 2) return false;
  return ((p[0] + p[1] + p[2] + col) & 1) == 0;
}

// Grid-stride over the cells of one colour (x-interior cells first); the
// component is a template parameter so every a == C decision folds at compile
// time.  (A grid-stride launch of about 24 blocks per SM measured faster than
// one thread per cell.)  CE: ef0 is the cell viscosity (CellEta), else the
// face arrays.
template <int D, typename T, int C, bool CE = false, bool PER = true>
__global__ void __launch_bounds__(256, CE ? 6 : 8) k_visc_smooth_c(T* __restrict__ u, const T* __restrict__ b, const T* ef0,
                                                      const T* ef1, const T* ef2, const __grid_constant__ Geom g, int col, T beta, int hom) {
  const int nt = rbx_count<D>(g);
  const T* ef[3] = {ef0, ef1, ef2};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    int p[3];
    if (!rbx_cell<D>(g, t, col, p)) continue;
    if (CE)
      visc_smooth_cell<D, T, C, PER>(u, b, CellEta<T>{ef0}, g, beta, hom, p);
    else
      visc_smooth_cell<D, T, C, PER>(u, b, FaceEta<T>{ef}, g, beta, hom, p);
  }
}

// out = u - beta L u, or r = b - (u - beta L u) when b != nullptr, for every
// component of cell p (flat index t).  Interior cells and wall cells are two
// separate branches (warps are almost always uniform).
template <int D, typename T, bool PER = true, typename EF>
__host__ __device__ __forceinline__ void visc_op_cell(const T* __restrict__ u, const T* __restrict__ b,
                                                     T* __restrict__ out, const EF& ef, const Geom& g, T beta,
                                                     int hom, const int* p, int t) {
  if (interior<D>(g, p)) {
    const Strides S = make_strides(g);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const size_t o = (size_t)c * g.ncell + t;
      const T Lu = tensor_interior<D, T>(u, ef, g, S, c, p);
      out[o] = op_out<T>(u[o], Lu, beta, b, o);
    }
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const size_t o = (size_t)c * g.ncell + t;
      const T Lu = mg_tensor_point<D, T, PER>(u, ef, g, c, p, hom != 0);
      out[o] = op_out<T>(u[o], Lu, beta, b, o);
    }
  }
}

template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_visc_op_at(const T* __restrict__ u, const T* __restrict__ b,
                                                     T* __restrict__ out, const T* ef0, const T* ef1, const T* ef2,
                                                     const Geom& g, T beta, int hom, int t) {
  const T* ef[3] = {ef0, ef1, ef2};
  int p[3];
  cell_coords<D>(g, t, p[0], p[1], p[2]);
  visc_op_cell<D, T, PER>(u, b, out, FaceEta<T>{ef}, g, beta, hom, p, t);
}

// out = u - beta L u, or r = b - (u - beta L u) when b != nullptr; one thread
// per cell, x-interior cells first (xi_cell), op3_blocks(g) blocks of 256.
// CE: ef0 is the cell viscosity (CellEta), else the face arrays.
template <int D, typename T, bool CE = false, bool PER = true>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (CE ? 4 : 5) : 4) k_visc_op3(const T* __restrict__ u, const T* __restrict__ b,
                                                 T* __restrict__ out, const T* ef0, const T* ef1, const T* ef2,
                                                 const __grid_constant__ Geom g, T beta, int hom) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p[3];
  if (t >= xi_count<D>(g) || !xi_cell<D>(g, t, p)) return;
  const T* ef[3] = {ef0, ef1, ef2};
  if (CE)
    visc_op_cell<D, T, PER>(u, b, out, CellEta<T>{ef0}, g, beta, hom, p, cidx<D>(g, p[0], p[1], p[2]));
  else
    visc_op_cell<D, T, PER>(u, b, out, FaceEta<T>{ef}, g, beta, hom, p, cidx<D>(g, p[0], p[1], p[2]));
}

template <int D>
inline unsigned op3_blocks(const Geom& g) {
  return (unsigned)((xi_count<D>(g) + 255) / 256);
}

// out = L_eta u (the stress divergence alone) at cell p; interior and wall
// cells in separate branches as in visc_op_cell
template <int D, typename T>
__host__ __device__ __forceinline__ void tensor_lu_cell(const T* __restrict__ u, T* __restrict__ out, const T* ef0,
                                                        const T* ef1, const T* ef2, const Geom& g, int hom,
                                                        const int* p) {
  const T* efa[3] = {ef0, ef1, ef2};
  const FaceEta<T> ef{efa};
  const int t = cidx<D>(g, p[0], p[1], p[2]);
  if (interior<D>(g, p)) {
    const Strides S = make_strides(g);
#pragma unroll
    for (int c = 0; c < D; ++c) out[(size_t)c * g.ncell + t] = tensor_interior<D, T>(u, ef, g, S, c, p);
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) out[(size_t)c * g.ncell + t] = mg_tensor_point<D, T>(u, ef, g, c, p, hom != 0);
  }
}

// the same at flat cell index t (row-major map)
template <int D, typename T>
__host__ __device__ __forceinline__ void k_tensor_lu_at(const T* __restrict__ u, T* __restrict__ out, const T* ef0,
                                                        const T* ef1, const T* ef2, const Geom& g, int hom, int t) {
  int p[3];
  cell_coords<D>(g, t, p[0], p[1], p[2]);
  tensor_lu_cell<D, T>(u, out, ef0, ef1, ef2, g, hom, p);
}

// grid-stride, x-interior cells first (xi_cell)
template <int D, typename T>
__global__ void __launch_bounds__(256) k_tensor_lu(const T* __restrict__ u, T* __restrict__ out, const T* ef0,
                                                  const T* ef1, const T* ef2, const __grid_constant__ Geom g, int hom) {
  const int nt = xi_count<D>(g);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    int p[3];
    if (xi_cell<D>(g, t, p)) tensor_lu_cell<D, T>(u, out, ef0, ef1, ef2, g, hom, p);
  }
}

// coarsest level: all sweeps in one block
template <int D, typename T>
__global__ void k_visc_bottom(T* __restrict__ u, const T* __restrict__ b, const T* ef0, const T* ef1,
                              const T* ef2, const __grid_constant__ Geom g, T beta, int nsweep, int hom) {
  const T* ef[3] = {ef0, ef1, ef2};
  int nt = rb_count<D>(g);
  for (int sw = 0; sw < nsweep; ++sw)
    for (int c = 0; c < D; ++c)
      for (int col = 0; col < 2; ++col) {
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
          int p[3];
          if (!rb_cell<D>(g, t, col, p)) continue;
          T v = visc_gs_point<D, T>(u, b, FaceEta<T>{ef}, g, c, p, beta, hom != 0);
          u[(size_t)c * g.ncell + cidx<D>(g, p[0], p[1], p[2])] = v;
        }
        __syncthreads();
      }
}

// ---------------------------------------------------------------------------
// cell-centred Poisson (MAC potential), Neumann walls
// ---------------------------------------------------------------------------
template <int D, typename T, bool PER = true>
__host__ __device__ inline T cell_gs_point(const T* __restrict__ x, const T* __restrict__ b, const Geom& g,
                                  const int* p) {
  T s = T(0);
  int cnt = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T lo = T(0), hi = T(0);
    const bool pa = PER && g.per[a];
    if (p[a] > 0 || pa) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = pa ? wrap_cell(q[a] - 1, g.n[a]) : q[a] - 1;
      lo = x[cidx<D>(g, q[0], q[1], q[2])];
      ++cnt;
    }
    if (p[a] < g.n[a] - 1 || pa) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = pa ? wrap_cell(q[a] + 1, g.n[a]) : q[a] + 1;
      hi = x[cidx<D>(g, q[0], q[1], q[2])];
      ++cnt;
    }
    s += lo + hi;
  }
  T hh = g_hh<T>(g);
  return (s - hh * b[cidx<D>(g, p[0], p[1], p[2])]) / T(cnt);
}

template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_cell_smooth_at(T* __restrict__ x, const T* __restrict__ b, const Geom& g, int col, int t) {
  int p[3];
  if (!rb_cell<D>(g, t, col, p)) return;
  x[cidx<D>(g, p[0], p[1], p[2])] = cell_gs_point<D, T, PER>(x, b, g, p);
}

template <int D, typename T, bool PER = true>
__global__ void k_cell_smooth(T* __restrict__ x, const T* __restrict__ b, const __grid_constant__ Geom g, int col) {
  int nt = rb_count<D>(g);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    k_cell_smooth_at<D, T, PER>(x, b, g, col, t);
  }
}

template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_cell_resid_at(const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, const Geom& g, int t) {
  const T ih = g_ih<T>(g);
  int p[3];
  cell_coords<D>(g, t, p[0], p[1], p[2]);
  T xc = x[t];
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T glo = T(0), ghi = T(0);
    const bool pa = PER && g.per[a];
    if (p[a] > 0 || pa) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = pa ? wrap_cell(q[a] - 1, g.n[a]) : q[a] - 1;
      glo = (xc - x[cidx<D>(g, q[0], q[1], q[2])]) * ih;
    }
    if (p[a] < g.n[a] - 1 || pa) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = pa ? wrap_cell(q[a] + 1, g.n[a]) : q[a] + 1;
      ghi = (x[cidx<D>(g, q[0], q[1], q[2])] - xc) * ih;
    }
    acc += (ghi - glo) * ih;
  }
  r[t] = b[t] - acc;
}

template <int D, typename T, bool PER = true>
__global__ void k_cell_resid(const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, const __grid_constant__ Geom g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_cell_resid_at<D, T, PER>(x, b, r, g, t);
  }
}

template <int D, typename T>
__global__ void k_cell_bottom(T* __restrict__ x, const T* __restrict__ b, const __grid_constant__ Geom g, int nsweep) {
  int nt = rb_count<D>(g);
  for (int sw = 0; sw < nsweep; ++sw)
    for (int col = 0; col < 2; ++col) {
      for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        int p[3];
        if (!rb_cell<D>(g, t, col, p)) continue;
        x[cidx<D>(g, p[0], p[1], p[2])] = cell_gs_point<D, T>(x, b, g, p);
      }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// nodal FE Poisson, Neumann walls
// ---------------------------------------------------------------------------
// stencil weight (times h^2) of offset o in {-1,0,1}^D
template <int D, typename T>
__host__ __device__ inline T fe_weight(int nz) {
  if (nz == 0) return T(-8.0 / 3.0);
  if (D == 2) return T(1.0 / 3.0);
  return nz == 1 ? T(0) : (nz == 2 ? T(1.0 / 6.0) : T(1.0 / 12.0));
}

// The kernels below take PER = false for a level with walls on every axis
// (the periodic wraps compile out; the code is then the plain reflection
// form) and PER = true otherwise.
template <int D, typename T, bool PER = true>
__host__ __device__ inline T nodal_lap_point(const T* __restrict__ x, const Geom& g, const int* p, bool skip_centre) {
  T s = T(0);
  const int K = D == 3 ? 27 : 9;
#pragma unroll
  for (int o = 0; o < K; ++o) {
    int oo[3];
    if (D == 3) {
      oo[0] = o / 9 - 1;
      oo[1] = (o / 3) % 3 - 1;
      oo[2] = o % 3 - 1;
    } else {
      oo[0] = o / 3 - 1;
      oo[1] = o % 3 - 1;
      oo[2] = 0;
    }
    int nz = (oo[0] != 0) + (oo[1] != 0) + (oo[2] != 0);
    if (nz == 0 && skip_centre) continue;
    if (D == 3 && nz == 1) continue;
    T w = fe_weight<D, T>(nz);
    s += w * ndget<D, T, PER>(x, g, p[0] + oo[0], p[1] + oo[1], p[2] + oo[2]);
  }
  return s;
}

template <int D>
__host__ __device__ inline bool mc_node(const Geom& g, int t, int col, int* p) {
  int e[3] = {g.n[0] + 1, g.n[1] + 1, D == 3 ? g.n[2] + 1 : 1};
  int cnt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int bit = (a < D) ? ((col >> a) & 1) : 0;
    cnt[a] = (a < D) ? (e[a] - bit + 1) / 2 : 1;
  }
  const int b0 = col & 1, b1 = (col >> 1) & 1;
  const int r = divm(t, cnt[0], g.m_mc0[b0]);
  const int i0 = t - r * cnt[0];
  const int i2 = divm(r, cnt[1], g.m_mc1[b1]);
  const int i1 = r - i2 * cnt[1];
  p[0] = 2 * i0 + (col & 1);
  p[1] = 2 * i1 + ((col >> 1) & 1);
  p[2] = D == 3 ? 2 * i2 + ((col >> 2) & 1) : 0;
  return i2 < cnt[2];
}

template <int D>
__host__ __device__ inline int mc_count(const Geom& g, int col) {
  int e[3] = {g.n[0] + 1, g.n[1] + 1, D == 3 ? g.n[2] + 1 : 1};
  int c = 1;
  for (int a = 0; a < D; ++a) c *= (e[a] - ((col >> a) & 1) + 1) / 2;
  return c;
}

template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_nodal_smooth_at(T* __restrict__ x, const T* __restrict__ b, const Geom& g, int col, int t) {
  int nt = mc_count<D>(g, col);
  const T hh = g_hh<T>(g);
  const T is0 = T(-3.0 / 8.0);  // 1 / centre weight
  
    int p[3];
    if (!mc_node<D>(g, t, col, p)) return;
    int id = nidx(g, p[0], p[1], p[2]);
    T s = nodal_lap_point<D, T, PER>(x, g, p, true);
    x[id] = (hh * b[id] - s) * is0;
  }

template <int D, typename T, bool PER = true>
__global__ void k_nodal_smooth(T* __restrict__ x, const T* __restrict__ b, const __grid_constant__ Geom g, int col) {
  int nt = mc_count<D>(g, col);
  const T hh = g_hh<T>(g);
  const T is0 = T(-3.0 / 8.0);  // 1 / centre weight
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    k_nodal_smooth_at<D, T, PER>(x, b, g, col, t);
  }
}

template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_nodal_resid_at(const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, const Geom& g, int t) {
  const T ihh = g_ihh<T>(g);
  
    int p[3];
    node_coords(g, t, p[0], p[1], p[2]);
    r[t] = b[t] - nodal_lap_point<D, T, PER>(x, g, p, false) * ihh;
  }

template <int D, typename T, bool PER = true>
__global__ void k_nodal_resid(const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, const __grid_constant__ Geom g) {
  const T ihh = g_ihh<T>(g);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.nnode; t += gridDim.x * blockDim.x) {
    k_nodal_resid_at<D, T, PER>(x, b, r, g, t);
  }
}

template <int D, typename T>
__global__ void k_nodal_bottom(T* __restrict__ x, const T* __restrict__ b, const __grid_constant__ Geom g, int nsweep) {
  const T hh = g_hh<T>(g);
  const T is0 = T(-3.0 / 8.0);
  const int ncol = 1 << D;
  for (int sw = 0; sw < nsweep; ++sw)
    for (int col = 0; col < ncol; ++col) {
      int nt = mc_count<D>(g, col);
      for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        int p[3];
        if (!mc_node<D>(g, t, col, p)) continue;
        int id = nidx(g, p[0], p[1], p[2]);
        T s = nodal_lap_point<D, T>(x, g, p, true);
        x[id] = (hh * b[id] - s) * is0;
      }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// transfers
// ---------------------------------------------------------------------------
// mean of the 2^D children, averaged axis by axis (x, then y, then z)
template <int D, typename T, bool SP = false>
__host__ __device__ __forceinline__ void k_restrict_cells_at(const T* __restrict__ f, T* __restrict__ c, const Geom& gf, const Geom& gc, int ncomp, long long tt) {
  
    int comp = 0;
    int t = (int)tt;
    while (t >= gc.ncell) {
      t -= gc.ncell;
      ++comp;
    }
    int I, J, K;
    cell_coords<D>(gc, t, I, J, K);
    const T* fc = f + (size_t)comp * gf.ncell;
    T v[2][2];
    for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk)
      for (int jj = 0; jj < 2; ++jj) {
        int j = 2 * J + jj, k = D == 3 ? 2 * K + kk : 0;
        v[kk][jj] = T(0.5) * (fc[lidx<D, SP>(gf, 2 * I, j, k)] + fc[lidx<D, SP>(gf, 2 * I + 1, j, k)]);
      }
    T w0 = T(0.5) * (v[0][0] + v[0][1]);
    T out = w0;
    if (D == 3) {
      T w1 = T(0.5) * (v[1][0] + v[1][1]);
      out = T(0.5) * (w0 + w1);
    }
    c[(size_t)comp * gc.ncell + t] = out;
  }

template <int D, typename T, bool SP = false>
__global__ void k_restrict_cells(const T* __restrict__ f, T* __restrict__ c, const __grid_constant__ Geom gf, const __grid_constant__ Geom gc, int ncomp) {
  long long tot = (long long)gc.ncell * ncomp;
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < tot;
       tt += (long long)gridDim.x * blockDim.x) {
    k_restrict_cells_at<D, T, SP>(f, c, gf, gc, ncomp, tt);
  }
}

// coarse a-face eta: mean of the fine a-faces tiling it (pairwise, axis order)
template <int D, typename T>
__host__ __device__ __forceinline__ void k_restrict_faces_at(const T* __restrict__ ff, T* __restrict__ fc, int a, const Geom& gf, const Geom& gc, int t) {
  
    int P[3];
    face_coords(gc, a, t, P[0], P[1], P[2]);
    // the two tangential axes in increasing order
    int o1 = -1, o2 = -1;
    for (int b = 0; b < D; ++b)
      if (b != a) {
        if (o1 < 0)
          o1 = b;
        else
          o2 = b;
      }
    T v[2][2];
    for (int s2 = 0; s2 < (D == 3 ? 2 : 1); ++s2)
      for (int s1 = 0; s1 < 2; ++s1) {
        int q[3] = {2 * P[0], 2 * P[1], D == 3 ? 2 * P[2] : 0};
        q[o1] += s1;
        if (D == 3) q[o2] += s2;
        v[s2][s1] = ff[fidx(gf, a, q[0], q[1], q[2])];
      }
    T w0 = T(0.5) * (v[0][0] + v[0][1]);
    T out = w0;
    if (D == 3) {
      T w1 = T(0.5) * (v[1][0] + v[1][1]);
      out = T(0.5) * (w0 + w1);
    }
    fc[t] = out;
  }

template <int D, typename T>
__global__ void k_restrict_faces(const T* __restrict__ ff, T* __restrict__ fc, int a, const __grid_constant__ Geom gf, const __grid_constant__ Geom gc) {
  int ex[3] = {gc.n[0] + (a == 0), gc.n[1] + (a == 1), gc.n[2] + (a == 2 && D == 3)};
  int nf = ex[0] * ex[1] * ex[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    k_restrict_faces_at<D, T>(ff, fc, a, gf, gc, t);
  }
}

// coarse cell value with ghost by reflection: sign -1 (Dirichlet error), +1 (Neumann)
template <int D, typename T, bool PER = true>
__host__ __device__ inline T cget_refl(const T* __restrict__ e, const Geom& g, int i, int j, int k, T sign) {
  T s = T(1);
  if (PER) {
    if (g.per[0]) i = wrap_cell(i, g.n[0]);
    if (g.per[1]) j = wrap_cell(j, g.n[1]);
    if (D == 3 && g.per[2]) k = wrap_cell(k, g.n[2]);
  }
  if (i < 0) { i = 0; s *= sign; }
  if (i >= g.n[0]) { i = g.n[0] - 1; s *= sign; }
  if (j < 0) { j = 0; s *= sign; }
  if (j >= g.n[1]) { j = g.n[1] - 1; s *= sign; }
  if (D == 3) {
    if (k < 0) { k = 0; s *= sign; }
    if (k >= g.n[2]) { k = g.n[2] - 1; s *= sign; }
  }
  return s * e[cidx<D>(g, i, j, k)];
}

// x_f += P e_c, cell-centred multilinear (3/4, 1/4 per axis), axis by axis
template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_prolong_cells_add_at(T* __restrict__ xf, const T* __restrict__ ec, const Geom& gf, const Geom& gc,
                                    int ncomp, T sign, long long tt) {
  
    int comp = 0;
    int t = (int)tt;
    while (t >= gf.ncell) {
      t -= gf.ncell;
      ++comp;
    }
    int i, j, k;
    cell_coords<D>(gf, t, i, j, k);
    const T* e = ec + (size_t)comp * gc.ncell;
    int I = i >> 1, J = j >> 1, K = k >> 1;
    int In = (i & 1) ? I + 1 : I - 1;
    int Jn = (j & 1) ? J + 1 : J - 1;
    int Kn = (k & 1) ? K + 1 : K - 1;
    T tz[2];
    for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk) {
      int kc = kk ? Kn : K;
      T ty[2];
      for (int jj = 0; jj < 2; ++jj) {
        int jc = jj ? Jn : J;
        ty[jj] = T(0.75) * cget_refl<D, T, PER>(e, gc, I, jc, kc, sign) +
                 T(0.25) * cget_refl<D, T, PER>(e, gc, In, jc, kc, sign);
      }
      tz[kk] = T(0.75) * ty[0] + T(0.25) * ty[1];
    }
    T v = D == 3 ? T(0.75) * tz[0] + T(0.25) * tz[1] : tz[0];
    xf[(size_t)comp * gf.ncell + t] += v;
  }

template <int D, typename T, bool PER = true>
__global__ void k_prolong_cells_add(T* __restrict__ xf, const T* __restrict__ ec, const __grid_constant__ Geom gf, const __grid_constant__ Geom gc,
                                    int ncomp, T sign) {
  long long tot = (long long)gf.ncell * ncomp;
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < tot;
       tt += (long long)gridDim.x * blockDim.x) {
    k_prolong_cells_add_at<D, T, PER>(xf, ec, gf, gc, ncomp, sign, tt);
  }
}

// The same prolongation with one thread per (coarse cell, component): the
// 3^D coarse neighbourhood is read once (with cget_refl's wraps, clamps and
// signs, which are exact: each sign is +-1) and each of the 2^D children is
// updated with the terms of k_prolong_cells_add_at in the same order.  Every
// level has even sizes (the hierarchy coarsens only even sizes), so each
// coarse cell has exactly 2^D children.
template <int D, typename T, bool PER = true, bool SP = false>
__host__ __device__ __forceinline__ void k_prolong_cells_add_c_at(T* __restrict__ xf, const T* __restrict__ ec,
                                                                  const Geom& gf, const Geom& gc, T sign,
                                                                  long long tt) {
  int comp = 0;
  int t = (int)tt;
  while (t >= gc.ncell) {
    t -= gc.ncell;
    ++comp;
  }
  int P[3];
  cell_coords<D>(gc, t, P[0], P[1], P[2]);
  const T* e = ec + (size_t)comp * gc.ncell;
  // per axis: coarse index and sign of the offsets -1, 0, +1
  int ix[3][3];
  T sg[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int q = (a < D) ? P[a] + d - 1 : 0;
      T s = T(1);
      if (a < D) {
        if (PER && gc.per[a]) q = wrap_cell(q, gc.n[a]);
        if (q < 0) {
          q = 0;
          s *= sign;
        }
        if (q >= gc.n[a]) {
          q = gc.n[a] - 1;
          s *= sign;
        }
      }
      ix[a][d] = q;
      sg[a][d] = s;
    }
  T v[D == 3 ? 3 : 1][3][3];
#pragma unroll
  for (int dz = 0; dz < (D == 3 ? 3 : 1); ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int kz = D == 3 ? dz : 0;
        const T s = sg[0][dx] * sg[1][dy] * (D == 3 ? sg[2][kz] : T(1));
        v[dz][dy][dx] = s * e[cidx<D>(gc, ix[0][dx], ix[1][dy], D == 3 ? ix[2][kz] : 0)];
      }
  T* x = xf + (size_t)comp * gf.ncell;
#pragma unroll
  for (int ck = 0; ck < (D == 3 ? 2 : 1); ++ck)
#pragma unroll
    for (int cj = 0; cj < 2; ++cj)
#pragma unroll
      for (int ci = 0; ci < 2; ++ci) {
        // child (2I + ci, 2J + cj, 2K + ck): its own coarse cell (offset 1)
        // and the neighbour on the child's side (offset 2 or 0)
        const int nx = ci ? 2 : 0, ny = cj ? 2 : 0, nz = D == 3 ? (ck ? 2 : 0) : 0;
        T tz[2];
#pragma unroll
        for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk) {
          const int kz = D == 3 ? (kk ? nz : 1) : 0;
          T ty[2];
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int jy = jj ? ny : 1;
            ty[jj] = T(0.75) * v[kz][jy][1] + T(0.25) * v[kz][jy][nx];
          }
          tz[kk] = T(0.75) * ty[0] + T(0.25) * ty[1];
        }
        const T val = D == 3 ? T(0.75) * tz[0] + T(0.25) * tz[1] : tz[0];
        x[lidx<D, SP>(gf, 2 * P[0] + ci, 2 * P[1] + cj, D == 3 ? 2 * P[2] + ck : 0)] += val;
      }
}

template <int D, typename T, bool PER = true, bool SP = false>
__global__ void k_prolong_cells_add_c(T* __restrict__ xf, const T* __restrict__ ec, const __grid_constant__ Geom gf,
                                      const __grid_constant__ Geom gc, int ncomp, T sign) {
  const long long tot = (long long)gc.ncell * ncomp;
  for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt < tot;
       tt += (long long)gridDim.x * blockDim.x)
    k_prolong_cells_add_c_at<D, T, PER, SP>(xf, ec, gf, gc, sign, tt);
}

// full weighting onto coarse nodes (even reflection), axis by axis
template <int D, typename T, bool PER = true>
__host__ __device__ __forceinline__ void k_restrict_nodes_at(const T* __restrict__ rf, T* __restrict__ rc, const Geom& gf, const Geom& gc, int t) {
  
    int I, J, K;
    node_coords(gc, t, I, J, K);
    T zr[3];
    for (int kk = 0; kk < (D == 3 ? 3 : 1); ++kk) {
      int k = D == 3 ? 2 * K + kk - 1 : 0;
      T yr[3];
      for (int jj = 0; jj < 3; ++jj) {
        int j = 2 * J + jj - 1;
        T cen = ndget<D, T, PER>(rf, gf, 2 * I, j, k);
        T lo = ndget<D, T, PER>(rf, gf, 2 * I - 1, j, k);
        T hi = ndget<D, T, PER>(rf, gf, 2 * I + 1, j, k);
        yr[jj] = T(0.5) * cen + T(0.25) * (lo + hi);
      }
      zr[kk] = T(0.5) * yr[1] + T(0.25) * (yr[0] + yr[2]);
    }
    rc[t] = D == 3 ? T(0.5) * zr[1] + T(0.25) * (zr[0] + zr[2]) : zr[0];
  }

template <int D, typename T, bool PER = true>
__global__ void k_restrict_nodes(const T* __restrict__ rf, T* __restrict__ rc, const __grid_constant__ Geom gf, const __grid_constant__ Geom gc) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < gc.nnode; t += gridDim.x * blockDim.x) {
    k_restrict_nodes_at<D, T, PER>(rf, rc, gf, gc, t);
  }
}

// x_f += P e_c, nodal multilinear, axis by axis
template <int D, typename T>
__host__ __device__ __forceinline__ void k_prolong_nodes_add_at(T* __restrict__ xf, const T* __restrict__ ec, const Geom& gf, const Geom& gc, int t) {
  
    int i, j, k;
    node_coords(gf, t, i, j, k);
    int I = i >> 1, J = j >> 1, K = k >> 1;
    T tz[2];
    for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk) {
      int kc = K + kk;
      if (D == 3 && kk == 1 && !(k & 1)) {
        tz[1] = T(0);
        continue;
      }
      T ty[2];
      for (int jj = 0; jj < 2; ++jj) {
        int jc = J + jj;
        if (jj == 1 && !(j & 1)) {
          ty[1] = T(0);
          continue;
        }
        T a0 = ec[nidx(gc, I, jc, D == 3 ? kc : 0)];
        ty[jj] = (i & 1) ? T(0.5) * (a0 + ec[nidx(gc, I + 1, jc, D == 3 ? kc : 0)]) : a0;
      }
      tz[kk] = (j & 1) ? T(0.5) * (ty[0] + ty[1]) : ty[0];
    }
    T v = (D == 3 && (k & 1)) ? T(0.5) * (tz[0] + tz[1]) : tz[0];
    xf[t] += v;
  }

template <int D, typename T>
__global__ void k_prolong_nodes_add(T* __restrict__ xf, const T* __restrict__ ec, const __grid_constant__ Geom gf, const __grid_constant__ Geom gc) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < gf.nnode; t += gridDim.x * blockDim.x) {
    k_prolong_nodes_add_at<D, T>(xf, ec, gf, gc, t);
  }
}

// ---------------------------------------------------------------------------
// exact coarsest-level solve: dense operator, Gauss-Jordan inverse, product
// ---------------------------------------------------------------------------
// cell Laplacian of x at p (Neumann walls), as k_cell_resid
template <int D, typename T>
__device__ inline T cell_lap_point(const T* __restrict__ x, const Geom& g, const int* p) {
  const T ih = g_ih<T>(g);
  const T xc = x[cidx<D>(g, p[0], p[1], p[2])];
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T glo = T(0), ghi = T(0);
    if (p[a] > 0 || g.per[a]) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = g.per[a] ? wrap_cell(q[a] - 1, g.n[a]) : q[a] - 1;
      glo = (xc - x[cidx<D>(g, q[0], q[1], q[2])]) * ih;
    }
    if (p[a] < g.n[a] - 1 || g.per[a]) {
      int q[3] = {p[0], p[1], p[2]};
      q[a] = g.per[a] ? wrap_cell(q[a] + 1, g.n[a]) : q[a] + 1;
      ghi = (x[cidx<D>(g, q[0], q[1], q[2])] - xc) * ih;
    }
    acc += (ghi - glo) * ih;
  }
  return acc;
}

// Column k of the bottom operator (kind 0 viscous, 1 MAC, 2 nodal), applied to
// the unit vector e_k held in X[k*n ..]; M is row-major with leading size ld.
// Singular problems get the constraint row/column of weights w (1 for cells,
// the dual-cell fraction for nodes).
template <int D>
__device__ inline void dense_build_col(int kind, double* __restrict__ X, double* __restrict__ M, int n, int ld,
                                       const double* ef0, const double* ef1, const double* ef2, const Geom& g, double beta,
                                       int k) {
  double* e = X + (size_t)k * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = (i == k) ? 1.0 : 0.0;
  __syncthreads();
  const double* ef[3] = {ef0, ef1, ef2};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v;
    int p[3];
    if (kind == 0) {
      const int c = i / g.ncell, t = i % g.ncell;
      cell_coords<D>(g, t, p[0], p[1], p[2]);
      v = e[i] - beta * mg_tensor_point<D, double>(e, FaceEta<double>{ef}, g, c, p, true);
    } else if (kind == 1) {
      cell_coords<D>(g, i, p[0], p[1], p[2]);
      v = cell_lap_point<D, double>(e, g, p);
    } else {
      const int e0 = g.n[0] + 1, e1 = g.n[1] + 1;
      p[0] = i % e0;
      p[1] = (i / e0) % e1;
      p[2] = i / (e0 * e1);
      v = nodal_lap_point<D, double>(e, g, p, false) * (1.0 / (g.h * g.h));
    }
    M[(size_t)i * ld + k] = v;
  }
  if (kind != 0 && threadIdx.x == 0) {
    // constraint entries of column k and (for the last block) the border
    double w = 1.0;
    if (kind == 2) {
      const int e0 = g.n[0] + 1, e1 = g.n[1] + 1;
      const int pi = k % e0, pj = (k / e0) % e1, pk = k / (e0 * e1);
      w = node_weight(g, pi, pj, pk, D);
    }
    M[(size_t)n * ld + k] = w;
    M[(size_t)k * ld + n] = w;
    if (k == 0) M[(size_t)n * ld + n] = 0.0;
  }
}

template <int D>
__global__ void k_dense_build(int kind, double* __restrict__ X, double* __restrict__ M, int n, int ld,
                              const double* ef0, const double* ef1, const double* ef2, const __grid_constant__ Geom g, double beta) {
  dense_build_col<D>(kind, X, M, n, ld, ef0, ef1, ef2, g, beta, blockIdx.x);
}

// Gauss-Jordan with partial pivoting on [M | I] (m x 2m, A), one block;
// writes the inverse to Minv (m x m).  Returns with Minv = 0 if singular.
__device__ inline void gauss_jordan_block(const double* __restrict__ M, int m, double* __restrict__ A,
                                          double* __restrict__ Minv) {
  __shared__ double fcol[kDenseMax + 1];
  __shared__ double sv[256];
  __shared__ int si[256];
  __shared__ int piv;
  const int w2 = 2 * m;
  for (int t = threadIdx.x; t < m * w2; t += blockDim.x) {
    const int i = t / w2, j = t % w2;
    A[t] = j < m ? M[(size_t)i * m + j] : (j - m == i ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) {
      const double a = fabs(A[(size_t)i * w2 + k]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int ib = k;
      for (int q = 0; q < (int)blockDim.x; ++q)
        if (sv[q] > b) {
          b = sv[q];
          ib = si[q];
        }
      piv = ib;
    }
    __syncthreads();
    const int pr = piv;
    if (pr != k)
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const double t0 = A[(size_t)k * w2 + j];
        A[(size_t)k * w2 + j] = A[(size_t)pr * w2 + j];
        A[(size_t)pr * w2 + j] = t0;
      }
    __syncthreads();
    const double d = A[(size_t)k * w2 + k];
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) A[(size_t)k * w2 + j] /= d;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) fcol[i] = A[(size_t)i * w2 + k];
    __syncthreads();
    for (int t = threadIdx.x; t < m * w2; t += blockDim.x) {
      const int i = t / w2, j = t % w2;
      if (i != k) A[t] -= fcol[i] * A[(size_t)k * w2 + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) Minv[t] = A[(size_t)(t / m) * w2 + m + t % m];
}

static __global__ void k_gauss_jordan(const double* __restrict__ M, int m, double* __restrict__ A, double* __restrict__ Minv) {
  gauss_jordan_block(M, m, A, Minv);
}

// x[i] = sum_j Minv[i][j] b[j] over the n unknowns (the bordered row/column,
// when present, multiplies a zero constraint value)
static __global__ void k_dense_apply(const double* __restrict__ Minv, int m, const double* __restrict__ b, int n,
                              double* __restrict__ x) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += Minv[(size_t)i * m + j] * b[j];
    x[i] = acc;
  }
}

}  // namespace hb
