// Device code of the explicit stages (Sec. III A-B), shared by the
// single-cavity launches (hb_explicit.cu) and the batched ones: per-element
// functions k_*_at and their grid-stride kernels.  Translation units that
// include it are compiled without FMA contraction (see hb_explicit.cu).
#pragma once
#include <cmath>
#include <cstring>

#include "hb_fp64bits.cuh"
#include "hb_internal.h"

namespace hb {

// The time-step constants of the explicit stages, rounded once on the host
// (the stages multiply by them where the plain formulas divide).
struct StepC {
  double dt;    // time step
  double dt2h;  // dt / (2h)
  double dth;   // dt / h
  double hdt;   // dt / 2
  double rho;   // density
  double irho;  // 1 / rho
  double dtr;   // dt / rho
  double idt;   // 1 / dt
  double inrm;  // 1 / (2^(D-1) h): the nodal divergence's normalisation
  double wl;    // 1 - theta: the weight of the explicit viscous term L_eta u^m
};

inline StepC step_consts(const Geom& g, int dim, double dt, double rho, double theta = 0.5) {
  StepC k;
  k.wl = 1.0 - theta;
  k.dt = dt;
  k.dt2h = dt / (2.0 * g.h);
  k.dth = dt / g.h;
  k.hdt = 0.5 * dt;
  k.rho = rho;
  k.irho = 1.0 / rho;
  k.dtr = dt / rho;
  k.idt = 1.0 / dt;
  k.inrm = 1.0 / ((double)(1 << (dim - 1)) * g.h);
  return k;
}

// ---------------------------------------------------------------------------
// Stage 1: strain rate and regularised viscosity (Eqs. 1, 21-23)
// ---------------------------------------------------------------------------
// g^(e2 / 2) for a half-integer exponent: products and one square root
// (within 2 ulp; pow, which the general exponent takes, costs several times
// as many FP64 instructions)
__host__ __device__ inline double half_pow(double g, int e2) {
  const int m = e2 < 0 ? -e2 : e2;
  double v = (m & 1) ? sqrt(g) : 1.0;
  for (int q = 0; q < (m >> 1); ++q) v *= g;
  return e2 < 0 ? 1.0 / v : v;
}

__host__ __device__ inline double viscosity(double g, const Rheo& r) {
  double x = r.m * g;
  double F;
  if (x < 1.0e-3) {
    // Taylor series of (1 - e^-x)/x, truncation below 1e-14 relative
    F = r.m * (1.0 - x / 2.0 + x * x / 6.0 - x * x * x / 24.0);
  } else {
    F = -expm1(-x) / g;
  }
  const bool half = r.e2 != kGeneralPow;
  if (r.reg_power) return (r.c2 * (half ? half_pow(g, r.e2) : pow(g, r.n)) + 0.5 * r.tau) * F;
  return r.c2 * (half ? half_pow(g, r.e2) : pow(g, r.n - 1.0)) + 0.5 * r.tau * F;
}

// |gamma_dot| = sqrt(1/2 tr(D D^T)) at cell t (Eq. 1), D = (grad u + grad u^T)/2
// from central differences with the wall ghosts
template <int D>
__host__ __device__ __forceinline__ double strain_norm_at(const double* __restrict__ u, const Geom& g, int t) {
  int i, j, k;
  cell_coords<D>(g, t, i, j, k);
  int p[3] = {i, j, k};
  double G[3][3];
  const double i2h = 0.5 * g.ih;  // 1/(2h), rounded once on the host
  // (grad u)_{ab} = d u_b / d x_a by central differences
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const double* ub = u + (size_t)b * g.ncell;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int q1[3] = {p[0], p[1], p[2]}, q0[3] = {p[0], p[1], p[2]};
      q1[a] += 1;
      q0[a] -= 1;
      G[a][b] = (uget<D>(ub, g, b, q1[0], q1[1], q1[2], false) -
                 uget<D>(ub, g, b, q0[0], q0[1], q0[2], false)) *
                i2h;
    }
  }
  // tr(D D^T) with D = (G + G^T)/2 symmetric: the diagonal D_aa = G_aa,
  // each off-diagonal pair counted twice
  double s = 0.0, so = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) s += G[a][a] * G[a][a];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = a + 1; b < D; ++b) {
      const double Dab = dhalf(G[a][b] + G[b][a]);
      so += Dab * Dab;
    }
  return sqrt(dhalf(s + dtwice(so)));
}

template <int D>
__host__ __device__ __forceinline__ void k_eta_at(const double* __restrict__ u, double* __restrict__ eta, const Geom& g, Rheo r, int t) {
  eta[t] = viscosity(strain_norm_at<D>(u, g, t), r);
}

template <int D>
__global__ void k_eta(const double* __restrict__ u, double* __restrict__ eta, const __grid_constant__ Geom g, Rheo r) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_eta_at<D>(u, eta, g, r, t);
  }
}

// face eta on level 0: mean of the two cells, wall faces take the interior cell
template <int D>
__host__ __device__ __forceinline__ void k_eta_faces_at(const double* __restrict__ eta, double* __restrict__ ef, int a, const Geom& g, int t) {
  
    int p[3];
    face_coords(g, a, t, p[0], p[1], p[2]);
    int L[3] = {p[0], p[1], p[2]}, R[3] = {p[0], p[1], p[2]};
    L[a] -= 1;
    if (g.per[a]) {  // periodic: the cells across the face, wrapped
      L[a] = wrap_cell(L[a], g.n[a]);
      R[a] = wrap_cell(R[a], g.n[a]);
    } else {
      if (L[a] < 0) L[a] = 0;
      if (R[a] >= g.n[a]) R[a] = g.n[a] - 1;
    }
    ef[t] = dhalf(eta[cidx<D>(g, L[0], L[1], L[2])] + eta[cidx<D>(g, R[0], R[1], R[2])]);
  }

template <int D>
__global__ void k_eta_faces(const double* __restrict__ eta, double* __restrict__ ef, int a, const __grid_constant__ Geom g) {
  int ex[3] = {g.n[0] + (a == 0), g.n[1] + (a == 1), g.n[2] + (a == 2 && D == 3)};
  int nf = ex[0] * ex[1] * ex[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    k_eta_faces_at<D>(eta, ef, a, g, t);
  }
}

// ---------------------------------------------------------------------------
// Stage 2: cell G p from nodes (L_eta u itself is evaluated by the
// multigrid unit's operator kernel, k_tensor_lu)
// ---------------------------------------------------------------------------
template <int D>
__host__ __device__ inline double grad_nodal(const double* __restrict__ p, const Geom& g, int a, int i, int j,
                                    int k) {
  // (p_+ - p_-)/h on each node pair along a, averaged over the other axes in order
  int c[3] = {i, j, k};
  double v[2][2];
  int o1 = -1, o2 = -1;
  for (int b = 0; b < D; ++b)
    if (b != a) {
      if (o1 < 0)
        o1 = b;
      else
        o2 = b;
    }
  for (int s1 = 0; s1 < 2; ++s1)
    for (int s2 = 0; s2 < (D == 3 ? 2 : 1); ++s2) {
      int q[3] = {c[0], c[1], c[2]};
      q[o1] += s1;
      if (D == 3) q[o2] += s2;
      int qh[3] = {q[0], q[1], q[2]};
      qh[a] += 1;
      v[s1][s2] = (p[nidx(g, qh[0], qh[1], qh[2])] - p[nidx(g, q[0], q[1], q[2])]) * g.ih;
    }
  if (D == 2) return dhalf(v[0][0] + v[1][0]);
  // average over o1 first, then o2
  double w0 = dhalf(v[0][0] + v[1][0]);
  double w1 = dhalf(v[0][1] + v[1][1]);
  return dhalf(w0 + w1);
}

template <int D>
__host__ __device__ __forceinline__ void k_grad_p_at(const double* __restrict__ p, double* __restrict__ Gp, const Geom& g, int t) {
  
    int i, j, k;
    cell_coords<D>(g, t, i, j, k);
#pragma unroll
    for (int a = 0; a < D; ++a) Gp[(size_t)a * g.ncell + t] = grad_nodal<D>(p, g, a, i, j, k);
  }

template <int D>
__global__ void k_grad_p(const double* __restrict__ p, double* __restrict__ Gp, const __grid_constant__ Geom g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_grad_p_at<D>(p, Gp, g, t);
  }
}

// ---------------------------------------------------------------------------
// Stage 3: Godunov edge states (Eqs. 11-14)
// ---------------------------------------------------------------------------
// Colella's slope from the five values w[0..4] at offsets -2..2
__host__ __device__ inline double slope5(const double* w) {
  double dlim[3], dC[3], df[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // cells p-1, p, p+1
    double dL = w[s + 1] - w[s];
    double dR = w[s + 2] - w[s + 1];
    dC[s] = dhalf(w[s + 2] - w[s]);
    // dL dR > 0 as a sign test (it differs from the product only where
    // |dL dR| underflows, below 1e-300, and then by less than 1e-150)
    dlim[s] = dsame_sign(dL, dR) ? dtwice(dminabs(dL, dR)) : 0.0;
    df[s] = dsgn_min(dC[s], dlim[s]);
  }
  double d4 = (4.0 / 3.0) * dC[1] - (1.0 / 6.0) * (df[2] + df[0]);
  return dsgn_min(d4, dlim[1]);
}

template <int D>
__host__ __device__ __forceinline__ void k_slopes_at(const double* __restrict__ u, double* __restrict__ slopes, const Geom& g, int t) {
  const int st[3] = {1, g.n[0], g.n[0] * g.n[1]};
  
    int p[3];
    cell_coords<D>(g, t, p[0], p[1], p[2]);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool inner = p[a] >= 2 && p[a] <= g.n[a] - 3;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double* uc = u + (size_t)c * g.ncell;
        double w[5];
        if (inner) {
#pragma unroll
          for (int o = -2; o <= 2; ++o) w[o + 2] = uc[t + o * st[a]];
        } else {
#pragma unroll
          for (int o = -2; o <= 2; ++o) {
            int q[3] = {p[0], p[1], p[2]};
            q[a] += o;
            w[o + 2] = uget<D>(uc, g, c, q[0], q[1], q[2], false);
          }
        }
        slopes[(size_t)(a * D + c) * g.ncell + t] = slope5(w);
      }
    }
  }

template <int D>
__global__ void k_slopes(const double* __restrict__ u, double* __restrict__ slopes, const __grid_constant__ Geom g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_slopes_at<D>(u, slopes, g, t);
  }
}

__host__ __device__ inline double riemann(double uL, double uR) {
  double s = uL + uR;
  if (dpos(uL) && dpos(s)) return uL;
  if (dneg(uR) && dneg(s)) return uR;
  return 0.0;
}

__host__ __device__ inline double upwind(double uL, double uR, double v) {
  if (dpos(v)) return uL;
  if (dneg(v)) return uR;
  return dhalf(uL + uR);
}

// Slope-only pre-states on the b-face between L and L+e_b (or wall values);
// st[c] returns the upwinded state of each component, vb the normal velocity.
template <int D>
__host__ __device__ inline void prestate_face(const double* __restrict__ u, const double* __restrict__ slopes,
                                     const Geom& g, const StepC& k, int b, const int* L, double* st,
                                     double& vb) {
  int Lw[3] = {L[0], L[1], L[2]};
  int R[3] = {L[0], L[1], L[2]};
  R[b] += 1;
  double sL[3], sR[3];
  if (g.per[b]) {
    R[b] = wrap_cell(R[b], g.n[b]);
    Lw[b] = wrap_cell(Lw[b], g.n[b]);
  }
  if (!g.per[b] && (L[b] < 0 || R[b] >= g.n[b])) {
    int side = L[b] < 0 ? 0 : 1;
#pragma unroll
    for (int c = 0; c < D; ++c) sL[c] = sR[c] = g.wu[b][side][c];
  } else {
    int tl = cidx<D>(g, Lw[0], Lw[1], Lw[2]), tr = cidx<D>(g, R[0], R[1], R[2]);
    double ubL = u[(size_t)b * g.ncell + tl], ubR = u[(size_t)b * g.ncell + tr];
    double facL = 0.5 - ubL * k.dt2h;
    double facR = 0.5 + ubR * k.dt2h;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      sL[c] = u[(size_t)c * g.ncell + tl] + facL * slopes[(size_t)(b * D + c) * g.ncell + tl];
      sR[c] = u[(size_t)c * g.ncell + tr] - facR * slopes[(size_t)(b * D + c) * g.ncell + tr];
    }
  }
  vb = riemann(sL[b], sR[b]);
#pragma unroll
  for (int c = 0; c < D; ++c) st[c] = (c == b) ? vb : upwind(sL[c], sR[c], vb);
}

struct Force {
  double f[3];
};

// The transverse terms hat_{bc} of the cell (Eq. 13), and from them the part of
// the cell's traces on its a-faces that does not depend on the face,
// tcom_{ac} = -dt/2 sum_{b != a} hat_{bc} + dt/2 F_c with F the cell's force
// (-G p [+ L_eta u] + f) / rho (Eq. 12).
template <int D>
__host__ __device__ __forceinline__ void k_hats_at(const double* __restrict__ u, const double* __restrict__ slopes,
                                                   const double* __restrict__ Gp, const double* __restrict__ Lu,
                                                   const Force& fo, int pv, double* __restrict__ hats,
                                                   double* __restrict__ tcom, const Geom& g, const StepC& k, int t) {
  int p[3];
  cell_coords<D>(g, t, p[0], p[1], p[2]);
  double hat[3][3];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    double stHi[3], stLo[3], vHi, vLo;
    prestate_face<D>(u, slopes, g, k, b, p, stHi, vHi);
    int Lm[3] = {p[0], p[1], p[2]};
    Lm[b] -= 1;
    prestate_face<D>(u, slopes, g, k, b, Lm, stLo, vLo);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      hat[b][c] = dhalf(vHi + vLo) * (stHi[c] - stLo[c]) * g.ih;
      hats[(size_t)(b * D + c) * g.ncell + t] = hat[b][c];
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const size_t o = (size_t)c * g.ncell + t;
    const double F = (-Gp[o] + (pv ? Lu[o] : 0.0) + fo.f[c]) * k.irho;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      // the sum over b != a in increasing b (with no leading 0.0 + : that
      // changes at most the sign of a zero sum, which no later step sees)
      const int b0 = a == 0 ? 1 : 0;
      double trans = hat[b0][c];
#pragma unroll
      for (int b = b0 + 1; b < D; ++b)
        if (b != a) trans += hat[b][c];
      tcom[(size_t)(a * D + c) * g.ncell + t] = -k.hdt * trans + k.hdt * F;
    }
  }
}

template <int D>
__global__ void k_hats(const double* __restrict__ u, const double* __restrict__ slopes,
                       const double* __restrict__ Gp, const double* __restrict__ Lu, Force fo, int pv,
                       double* __restrict__ hats, double* __restrict__ tcom, const __grid_constant__ Geom g,
                       const StepC k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_hats_at<D>(u, slopes, Gp, Lu, fo, pv, hats, tcom, g, k, t);
  }
}

// one-sided extrapolation of component c from cell q to its face along a,
// side = -1 (left state: face above q) or +1 (right state: face below q)
template <int D>
__host__ __device__ inline double trace(const double* __restrict__ u, const double* __restrict__ slopes,
                                        const double* __restrict__ tcom, const Geom& g, const StepC& k, int a, int c,
                                        int tq, bool left) {
  double common = tcom[(size_t)(a * D + c) * g.ncell + tq];
  double ua = u[(size_t)a * g.ncell + tq];
  double s = slopes[(size_t)(a * D + c) * g.ncell + tq];
  double uc = u[(size_t)c * g.ncell + tq];
  if (left) {
    double fac = 0.5 - ua * k.dt2h;
    return uc + fac * s + common;
  }
  double fac = 0.5 + ua * k.dt2h;
  return uc - fac * s + common;
}

template <int D>
__host__ __device__ __forceinline__ void k_traces_at(const double* __restrict__ u, const double* __restrict__ slopes,
                         const double* __restrict__ tcom, int a,
                         double* __restrict__ uL, double* __restrict__ uR, double* __restrict__ uadv,
                         const Geom& g, const StepC& k, int t) {
  int ex[3] = {g.n[0] + (a == 0), g.n[1] + (a == 1), g.n[2] + (a == 2 && D == 3)};
  int nf = ex[0] * ex[1] * ex[2];
  
    int R[3];
    face_coords(g, a, t, R[0], R[1], R[2]);
    int L[3] = {R[0], R[1], R[2]};
    L[a] -= 1;
    if (g.per[a]) {  // periodic: the cells across the face, wrapped (face n repeats face 0)
      L[a] = wrap_cell(L[a], g.n[a]);
      R[a] = wrap_cell(R[a], g.n[a]);
    } else if (L[a] < 0 || R[a] >= g.n[a]) {
      int side = L[a] < 0 ? 0 : 1;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        uL[(size_t)c * nf + t] = g.wu[a][side][c];
        uR[(size_t)c * nf + t] = g.wu[a][side][c];
      }
      uadv[t] = 0.0;
      return;
    }
    int tl = cidx<D>(g, L[0], L[1], L[2]), tr = cidx<D>(g, R[0], R[1], R[2]);
    double vl = 0, vr = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double l = trace<D>(u, slopes, tcom, g, k, a, c, tl, true);
      double rr = trace<D>(u, slopes, tcom, g, k, a, c, tr, false);
      uL[(size_t)c * nf + t] = l;
      uR[(size_t)c * nf + t] = rr;
      if (c == a) {
        vl = l;
        vr = rr;
      }
    }
    uadv[t] = riemann(vl, vr);
  }

template <int D>
__global__ void k_traces(const double* __restrict__ u, const double* __restrict__ slopes,
                         const double* __restrict__ tcom, int a,
                         double* __restrict__ uL, double* __restrict__ uR, double* __restrict__ uadv,
                         const __grid_constant__ Geom g, const StepC k) {
  int ex[3] = {g.n[0] + (a == 0), g.n[1] + (a == 1), g.n[2] + (a == 2 && D == 3)};
  int nf = ex[0] * ex[1] * ex[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    k_traces_at<D>(u, slopes, tcom, a, uL, uR, uadv, g, k, t);
  }
}

// ---------------------------------------------------------------------------
// Stage 4: MAC divergence and correction
// ---------------------------------------------------------------------------
template <int D>
__host__ __device__ __forceinline__ void k_mac_rhs_at(const double* ua0, const double* ua1, const double* ua2,
                          double* __restrict__ rhs, const Geom& g, int t) {
  const double* ua[3] = {ua0, ua1, ua2};
  
    int p[3];
    cell_coords<D>(g, t, p[0], p[1], p[2]);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int q[3] = {p[0], p[1], p[2]};
      double lo = ua[a][fidx(g, a, q[0], q[1], q[2])];
      q[a] += 1;
      double hi = ua[a][fidx(g, a, q[0], q[1], q[2])];
      acc += (hi - lo) * g.ih;
    }
    rhs[t] = acc;
  }

template <int D>
__global__ void k_mac_rhs(const double* ua0, const double* ua1, const double* ua2,
                          double* __restrict__ rhs, const __grid_constant__ Geom g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_mac_rhs_at<D>(ua0, ua1, ua2, rhs, g, t);
  }
}

template <int D>
__host__ __device__ __forceinline__ void k_mac_correct_at(const double* __restrict__ uadv, const double* __restrict__ phi,
                              double* __restrict__ umac, int a, const Geom& g, int t) {
  
    int R[3];
    face_coords(g, a, t, R[0], R[1], R[2]);
    if (!g.per[a] && (R[a] == 0 || R[a] == g.n[a])) {
      umac[t] = 0.0;
      return;
    }
    int L[3] = {R[0], R[1], R[2]};
    L[a] -= 1;
    if (g.per[a]) {
      L[a] = wrap_cell(L[a], g.n[a]);
      R[a] = wrap_cell(R[a], g.n[a]);
    }
    double gr = (phi[cidx<D>(g, R[0], R[1], R[2])] - phi[cidx<D>(g, L[0], L[1], L[2])]) * g.ih;
    umac[t] = uadv[t] - gr;
  }

template <int D>
__global__ void k_mac_correct(const double* __restrict__ uadv, const double* __restrict__ phi,
                              double* __restrict__ umac, int a, const __grid_constant__ Geom g) {
  int ex[3] = {g.n[0] + (a == 0), g.n[1] + (a == 1), g.n[2] + (a == 2 && D == 3)};
  int nf = ex[0] * ex[1] * ex[2];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += gridDim.x * blockDim.x) {
    k_mac_correct_at<D>(uadv, phi, umac, a, g, t);
  }
}

// ---------------------------------------------------------------------------
// Stage 5: upwinding with u^MAC, convective term, viscous right-hand side
// ---------------------------------------------------------------------------
template <int D>
__host__ __device__ __forceinline__ void k_advect_rhs_at(const double* __restrict__ u, const double* uL0, const double* uL1,
                             const double* uL2, const double* uR0, const double* uR1,
                             const double* uR2, const double* um0, const double* um1,
                             const double* um2, const double* __restrict__ Gp,
                             const double* __restrict__ Lu, Force fo,
                             double* __restrict__ rhs, const Geom& g, const StepC& k, int t) {
  const double* uL[3] = {uL0, uL1, uL2};
  const double* uR[3] = {uR0, uR1, uR2};
  const double* um[3] = {um0, um1, um2};
  
    int p[3];
    cell_coords<D>(g, t, p[0], p[1], p[2]);
    double A[3] = {0.0, 0.0, 0.0};  // h times the convective term (1/h goes into dt/h)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int nf = g.nface[a];
      int q[3] = {p[0], p[1], p[2]};
      int flo = fidx(g, a, q[0], q[1], q[2]);
      q[a] += 1;
      int fhi = fidx(g, a, q[0], q[1], q[2]);
      double vlo = um[a][flo], vhi = um[a][fhi];
      double vbar = dhalf(vhi + vlo);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double thi = upwind(uL[a][(size_t)c * nf + fhi], uR[a][(size_t)c * nf + fhi], vhi);
        double tlo = upwind(uL[a][(size_t)c * nf + flo], uR[a][(size_t)c * nf + flo], vlo);
        A[c] += vbar * (thi - tlo);
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      size_t o = (size_t)c * g.ncell + t;
      const double lw = k.wl == 0.5 ? dhalf(Lu[o]) : k.wl * Lu[o];  // (1 - theta) L_eta u^m
      rhs[o] = u[o] - k.dth * A[c] + k.dtr * (-Gp[o] + lw + fo.f[c]);
    }
  }

template <int D>
__global__ void k_advect_rhs(const double* __restrict__ u, const double* uL0, const double* uL1,
                             const double* uL2, const double* uR0, const double* uR1,
                             const double* uR2, const double* um0, const double* um1,
                             const double* um2, const double* __restrict__ Gp,
                             const double* __restrict__ Lu, Force fo,
                             double* __restrict__ rhs, const __grid_constant__ Geom g, const StepC k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_advect_rhs_at<D>(u, uL0, uL1, uL2, uR0, uR1, uR2, um0, um1, um2, Gp, Lu, fo, rhs, g, k, t);
  }
}

// ---------------------------------------------------------------------------
// Stage 7: nodal divergence of u*/dt + G p/rho, projection update
// ---------------------------------------------------------------------------
// G p of the cell from the nodes, and the cell field the nodal divergence
// takes, w = u*/dt + (G p)/rho, formed once per cell instead of at each of
// the cell's 2^D nodes
template <int D>
__host__ __device__ __forceinline__ void k_grad_p_w_at(const double* __restrict__ p, const double* __restrict__ ustar,
                                                       double* __restrict__ Gp, double* __restrict__ w, const Geom& g,
                                                       const StepC& k, int t) {
  int i, j, kk;
  cell_coords<D>(g, t, i, j, kk);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const size_t o = (size_t)a * g.ncell + t;
    const double gp = grad_nodal<D>(p, g, a, i, j, kk);
    Gp[o] = gp;
    w[o] = ustar[o] * k.idt + gp * k.irho;
  }
}

template <int D>
__global__ void k_grad_p_w(const double* __restrict__ p, const double* __restrict__ ustar, double* __restrict__ Gp,
                           double* __restrict__ w, const __grid_constant__ Geom g, const StepC k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_grad_p_w_at<D>(p, ustar, Gp, w, g, k, t);
  }
}

// the nodal right-hand side: the divergence of w over the node's 2^D cells
template <int D>
__host__ __device__ __forceinline__ void k_nodal_rhs_at(const double* __restrict__ w, double* __restrict__ out,
                                                        const Geom& g, const StepC& k, int t) {
  
    int p[3];
    node_coords(g, t, p[0], p[1], p[2]);
    double acc = 0.0;
    const int ncorner = D == 3 ? 8 : 4;
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
      for (int cn = 0; cn < ncorner; ++cn) {
        // corner bits, last axis fastest (lexicographic order)
        int cb[3];
        if (D == 3) {
          cb[0] = (cn >> 2) & 1;
          cb[1] = (cn >> 1) & 1;
          cb[2] = cn & 1;
        } else {
          cb[0] = (cn >> 1) & 1;
          cb[1] = cn & 1;
          cb[2] = 1;
        }
        int q[3] = {p[0] - 1 + cb[0], p[1] - 1 + cb[1], D == 3 ? p[2] - 1 + cb[2] : 0};
#pragma unroll
        for (int b = 0; b < D; ++b)
          if (g.per[b]) q[b] = wrap_cell(q[b], g.n[b]);
        bool in = q[0] >= 0 && q[0] < g.n[0] && q[1] >= 0 && q[1] < g.n[1] &&
                  (D == 2 || (q[2] >= 0 && q[2] < g.n[2]));
        if (!in) continue;
        const double v = w[(size_t)a * g.ncell + cidx<D>(g, q[0], q[1], q[2])];
        acc += cb[a] ? v : -v;
      }
    }
    // 1 / (w 2^(D-1) h) with w the node's weight (1/2 per wall axis): the
    // power of two 1/w is exact
    double iw = 1.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (!g.per[a] && (p[a] == 0 || p[a] == g.n[a])) iw *= 2.0;
    out[t] = k.rho * (acc * (iw * k.inrm));
  }

template <int D>
__global__ void k_nodal_rhs(const double* __restrict__ w, double* __restrict__ out, const __grid_constant__ Geom g,
                            const StepC k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.nnode; t += gridDim.x * blockDim.x) {
    k_nodal_rhs_at<D>(w, out, g, k, t);
  }
}

template <int D>
__host__ __device__ __forceinline__ void k_project_update_at(double* __restrict__ u, const double* __restrict__ Gp,
                                 const double* __restrict__ phi, const Geom& g, const StepC& sc, int t) {
  
    int i, j, k;
    cell_coords<D>(g, t, i, j, k);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      size_t o = (size_t)a * g.ncell + t;
      double gphi = grad_nodal<D>(phi, g, a, i, j, k);
      u[o] = u[o] + sc.dtr * (Gp[o] - gphi);
    }
  }

template <int D>
__global__ void k_project_update(double* __restrict__ u, const double* __restrict__ Gp,
                                 const double* __restrict__ phi, const __grid_constant__ Geom g, const StepC k) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell; t += gridDim.x * blockDim.x) {
    k_project_update_at<D>(u, Gp, phi, g, k, t);
  }
}

}  // namespace hb
