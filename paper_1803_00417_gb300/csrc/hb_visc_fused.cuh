// One red-black Gauss-Seidel sweep of one velocity component of the tensor
// viscous operator (I - beta L_eta) u = b in a single launch, for the FP32
// finest level of the viscous V-cycles in 3D (cell viscosity; the same
// per-cell update as k_visc_smooth_c<3, float, C, true>: red cells, those with
// i + j + k even, from the old values, then black cells from the new red
// ones).
//
// The two colour launches of k_visc_smooth_c read u_c, the two other
// components, the viscosity and b_c once each per colour (18 B/cell, twice);
// this kernel reads each of them once and writes u_c once (24 B/cell for the
// whole sweep).  A block owns a tile of TX x TY cells of every z plane in a
// chunk of ZC planes and marches along z with the planes staged in shared
// memory (four plane slots, a ring of two cells around the tile):
//   step r: stage plane r+1; update the red cells of plane r on the tile and
//   its one-cell ring (the ring's red values belong to neighbouring tiles;
//   recomputing them here from the same inputs gives the same values); update
//   the black cells of plane r-1 from the new red values of planes r-2..r and
//   write plane r-1 (both colours) out.
// Because neighbouring tiles read the old values of cells this tile writes,
// the sweep writes to a second array; the caller swaps the two after each
// component (an even number of sweeps ends in the original array).
// Wall cells take the general stencil with the reflected ghosts of the
// point update, reading the staged in-domain values.
#pragma once
#include "hb_common.cuh"

namespace hb {
namespace fused {

constexpr int TX = 32, TY = 16;              // interior columns of a tile
constexpr int EX = TX + 4, EY = TY + 4;      // with a ring of two cells
constexpr int EP = EX * EY;
constexpr int RX = TX + 2, RY = TY + 2;      // the red region: tile + one cell
constexpr int RP = RX * RY;
constexpr int ZC = 16;                       // z planes per block
constexpr int NT = 256;

struct Smem {
  float u[4][EP];  // u_c: old values, red cells overwritten by the new ones
  float a[4][EP];  // the first other component
  float b[4][EP];  // the second other component
  float e[4][EP];  // the cell viscosity
  float r[4][RP];  // b_c over the red region
};

template <int C>
struct Tile {
  Smem& s;
  int x0, y0;
  const Geom& g;
  __device__ int at(int gx, int gy) const { return (gy - y0 + 2) * EX + (gx - x0 + 2); }
  // component q at an in-domain cell
  __device__ float comp(int q, int gx, int gy, int gz) const {
    const int sl = gz & 3, i = at(gx, gy);
    if (q == C) return s.u[sl][i];
    return q == (C == 0 ? 1 : 0) ? s.a[sl][i] : s.b[sl][i];
  }
  __device__ float eta(int gx, int gy, int gz) const { return s.e[gz & 3][at(gx, gy)]; }
  // component q at cell p with at most axis ax outside the domain (odd
  // reflection about the wall value, as uget_axis)
  __device__ float comp_axis(int q, int* p, int ax, bool hom) const {
    int side = -1;
    const int keep = p[ax];
    if (p[ax] < 0) {
      side = 0;
      p[ax] = -p[ax] - 1;
    } else if (p[ax] >= g.n[ax]) {
      side = 1;
      p[ax] = 2 * g.n[ax] - 1 - p[ax];
    }
    const float v = comp(q, p[0], p[1], p[2]);
    p[ax] = keep;
    if (side < 0) return v;
    const float ub = hom ? 0.f : g.fwu[ax][side][q];
    return 2.f * ub - v;
  }
  // the face viscosity of axis a whose upper cell is q: mean of the two cells,
  // a wall face takes the interior cell (CellEta::at)
  __device__ float face_eta(int a, const int* q) const {
    int L[3] = {q[0], q[1], q[2]}, R[3] = {q[0], q[1], q[2]};
    L[a] = q[a] > 0 ? q[a] - 1 : 0;
    R[a] = q[a] < g.n[a] ? q[a] : g.n[a] - 1;
    return 0.5f * (eta(L[0], L[1], L[2]) + eta(R[0], R[1], R[2]));
  }
  // mg_face_cross: mean of the two cells' central c-differences of component a
  // on the a-face above cell L
  __device__ float face_cross(int a, int c, const int* L, bool hom) const {
    if (L[a] < 0 || L[a] >= g.n[a] - 1) return 0.f;
    int p1[3] = {L[0], L[1], L[2]}, p0[3] = {L[0], L[1], L[2]};
    p1[c] += 1;
    p0[c] -= 1;
    const float dL = comp_axis(a, p1, c, hom) - comp_axis(a, p0, c, hom);
    p1[a] += 1;
    p0[a] += 1;
    const float dR = comp_axis(a, p1, c, hom) - comp_axis(a, p0, c, hom);
    return (dL + dR) * g.fq4;
  }

  // visc_gs_interior<3, float, CellEta> on the staged planes
  __device__ float interior(int gx, int gy, int gz, float bval, float beta) const {
    const int i0 = at(gx, gy);
    const int zm = (gz - 1) & 3, z0 = gz & 3, zp = (gz + 1) & 3;
    const float bs = beta * (g.fihh * 0.5f);
    const float ec = s.e[z0][i0];
    float elo[3], ehi[3];
    elo[0] = s.e[z0][i0 - 1] + ec;
    ehi[0] = ec + s.e[z0][i0 + 1];
    elo[1] = s.e[z0][i0 - EX] + ec;
    ehi[1] = ec + s.e[z0][i0 + EX];
    elo[2] = s.e[zm][i0] + ec;
    ehi[2] = ec + s.e[zp][i0];
    const float* u0 = s.u[z0];
    float ulo[3] = {u0[i0 - 1], u0[i0 - EX], s.u[zm][i0]};
    float uhi[3] = {u0[i0 + 1], u0[i0 + EX], s.u[zp][i0]};
    float offd = 0.f, diag = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float kappa = (a == C) ? 2.f : 1.f;
      offd += kappa * (elo[a] * ulo[a] + ehi[a] * uhi[a]);
      diag += kappa * (elo[a] + ehi[a]);
    }
    float cross = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == C) continue;
      const float(*A)[EP] = a == (C == 0 ? 1 : 0) ? s.a : s.b;
      // value of component a at offset (da along a) + (dc along C)
      auto v = [&](int da, int dc) {
        int d[3] = {0, 0, 0};
        d[a] += da;
        d[C] += dc;
        return A[(gz + d[2]) & 3][i0 + d[0] + EX * d[1]];
      };
      const float mid = v(0, 1) - v(0, -1);
      const float xhi = mid + (v(1, 1) - v(1, -1));
      const float xlo = (v(-1, 1) - v(-1, -1)) + mid;
      cross += ehi[a] * xhi - elo[a] * xlo;
    }
    return (bval + bs * (offd + 0.25f * cross)) / (1.f + bs * diag);
  }

  // visc_gs_point<3, float, CellEta> on the staged planes
  __device__ float wall(int gx, int gy, int gz, float bval, float beta, bool hom) const {
    const int p[3] = {gx, gy, gz};
    const float ih = g.fih, ihh = g.fihh;
    float offd = 0.f, diag = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float kappa = (a == C) ? 2.f : 1.f;
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        int q[3] = {p[0], p[1], p[2]};
        int fq[3] = {p[0], p[1], p[2]};
        if (sd == 0) {
          q[a] -= 1;
        } else {
          q[a] += 1;
          fq[a] += 1;
        }
        const float wf = kappa * face_eta(a, fq) * ihh;
        const bool w = (sd == 0) ? (p[a] == 0) : (p[a] == g.n[a] - 1);
        if (w) {
          const float ub = hom ? 0.f : g.fwu[a][sd][C];
          offd += 2.f * wf * ub;
          diag += 2.f * wf;
        } else {
          offd += wf * comp(C, q[0], q[1], q[2]);
          diag += wf;
        }
      }
    }
    float cross = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == C) continue;
      int Llo[3] = {p[0], p[1], p[2]};
      Llo[a] -= 1;
      int fhi[3] = {p[0], p[1], p[2]};
      fhi[a] += 1;
      const float fluxhi = face_eta(a, fhi) * face_cross(a, C, p, hom);
      const float fluxlo = face_eta(a, p) * face_cross(a, C, Llo, hom);
      cross += (fluxhi - fluxlo) * ih;
    }
    return (bval + beta * (offd + cross)) / (1.f + beta * diag);
  }

  __device__ float update(int gx, int gy, int gz, float bval, float beta, bool hom) const {
    const bool in = gx >= 1 && gx <= g.n[0] - 2 && gy >= 1 && gy <= g.n[1] - 2 && gz >= 1 && gz <= g.n[2] - 2;
    return in ? interior(gx, gy, gz, bval, beta) : wall(gx, gy, gz, bval, beta, hom);
  }
};

// uc, ua, ub: component C and the other two components in increasing order;
// bc: component C of the right-hand side; out: component C after the sweep
template <int C>
__global__ void __launch_bounds__(NT, 4) k_visc_sweep_rb(const float* __restrict__ uc, const float* __restrict__ ua,
                                                        const float* __restrict__ ub, const float* __restrict__ eta,
                                                        const float* __restrict__ bc, float* __restrict__ out,
                                                        const __grid_constant__ Geom g, float beta, int hom) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
  const int z1 = min(z0 + ZC, nz);
  const Tile<C> T{s, x0, y0, g};
  const bool hm = hom != 0;

  auto stage = [&](int kz) {  // plane kz over the tile and its two-cell ring
    if (kz < 0 || kz >= nz) return;
    const int sl = kz & 3;
    const size_t plane = (size_t)nx * ny * kz;
    for (int q = threadIdx.x; q < EP; q += NT) {
      const int ey = q / EX, ex = q - ey * EX;
      const int gx = x0 - 2 + ex, gy = y0 - 2 + ey;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
      const size_t id = plane + gx + (size_t)nx * gy;
      s.u[sl][q] = uc[id];
      s.a[sl][q] = ua[id];
      s.b[sl][q] = ub[id];
      s.e[sl][q] = eta[id];
      if (ex >= 1 && ex <= RX && ey >= 1 && ey <= RY) s.r[sl][(ey - 1) * RX + (ex - 1)] = bc[id];
    }
  };

  stage(z0 - 2);
  stage(z0 - 1);
  stage(z0);
  for (int r = z0 - 1; r <= z1; ++r) {
    stage(r + 1);  // overwrites plane r - 3, no longer read
    __syncthreads();
    // red cells (i + j + k even) of plane r over the tile and its ring
    if (r >= 0 && r < nz) {
      const int sr = r & 3;
      for (int q = threadIdx.x; q < RY * (RX / 2); q += NT) {
        const int ry = q / (RX / 2), m = q - ry * (RX / 2);
        const int gy = y0 - 1 + ry;
        const int gx = x0 - 1 + 2 * m + ((x0 - 1 + gy + r) & 1);
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
        const float bval = s.r[sr][ry * RX + (gx - x0 + 1)];
        const float v = T.update(gx, gy, r, bval, beta, hm);
        s.u[r & 3][T.at(gx, gy)] = v;
      }
    }
    __syncthreads();
    // black cells of plane r - 1 over the tile; write the plane out
    const int k = r - 1;
    if (k >= z0 && k < z1) {
      const int sr = k & 3;
      for (int q = threadIdx.x; q < TY * (TX / 2); q += NT) {
        const int ty = q / (TX / 2), m = q - ty * (TX / 2);
        const int gy = y0 + ty;
        const int gxe = x0 + 2 * m;  // the pair (gxe, gxe + 1): one red, one black
        if (gy >= ny || gxe >= nx) continue;
        const bool first_black = ((gxe + gy + k) & 1) != 0;
        const int gb = first_black ? gxe : gxe + 1;
        float vb = 0.f;
        if (gb < nx) vb = T.update(gb, gy, k, s.r[sr][(gy - y0 + 1) * RX + (gb - x0 + 1)], beta, hm);
        const float vr0 = s.u[k & 3][T.at(gxe, gy)];
        const size_t id = gxe + (size_t)nx * (gy + (size_t)ny * k);
        if (gxe + 1 < nx) {
          const float vr1 = s.u[k & 3][T.at(gxe + 1, gy)];
          out[id] = first_black ? vb : vr0;
          out[id + 1] = first_black ? vr1 : vb;
        } else {
          out[id] = first_black ? vb : vr0;
        }
      }
    }
    __syncthreads();
  }
}

inline dim3 sweep_grid(const Geom& g) {
  return dim3((unsigned)((g.n[0] + TX - 1) / TX), (unsigned)((g.n[1] + TY - 1) / TY),
              (unsigned)((g.n[2] + ZC - 1) / ZC));
}

}  // namespace fused
}  // namespace hb
