// Finest-level FP32 viscous kernels (Eq. 16, face viscosities formed from the
// cell viscosity) with their operands staged in shared memory by the tensor
// memory accelerator (3D only): the red-black Gauss-Seidel sweep of one
// velocity component and one colour, and the operator u - beta L u (or the
// residual b - (u - beta L u)) of all three components.
//
// A block owns a tile of TX x TY cells in x, y and a chunk of TZ planes in z,
// and streams the planes z0 - 1 .. z0 + TZ through a ring of NS stages
// (stream_planes): one thread issues, per plane, cp.async.bulk.tensor loads of
// the three velocity components and the cell viscosity over the tile with a
// halo of kHX cells in x and one row in y (and, for the sweep, the right-hand
// side of the component over the tile) that complete on the stage's mbarrier,
// while the block works on the plane two stages behind.  A load's x
// coordinate is a multiple of 4 floats (16 bytes): the x halo is 4 cells so
// that x0 - 4 stays aligned.  Coordinates outside the grid read zeros, which
// only cells that take the global path below would see.
//
// Within a sweep of one colour, every value the update reads (u_c of the
// other colour, the other components, eta, b) is left unchanged by the sweep;
// the operator writes another array than it reads.  So stale or fresh copies
// are the same and the staged planes never need refreshing.  Interior cells
// run visc_gs_core / tensor_core on the values that visc_gs_interior /
// tensor_interior gather: the results are the same bit for bit as those of
// k_visc_smooth_c / k_visc_op3.  Cells on a y or z wall take the global path
// inside the tile; the cells on the two x walls, whose warps would otherwise
// run the wall stencil next to interior cells, are taken by kWallRows-row wall
// blocks placed after the tiles of each z chunk, so that they run while that
// chunk's planes are still in L2.  Walls on every axis (the wall-only forms).
//
// Every mbarrier wait is bounded (kStageWait polls).  A block that gives up
// sets *err, stops working, waits (bounded again) for the loads it has in
// flight so that no copy is still writing its shared memory, and exits; the
// host reports HBF_ERR_TIMEOUT after the solve.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "hb_mg_kernels.cuh"

namespace hb {
namespace tma {

constexpr int kHX = 4;            // x halo: 16 bytes of floats
constexpr int kThreads = 256;
constexpr int kWallRows = 256;    // rows per x-wall block (one thread per row)
constexpr long long kStageWait = 1 << 20;
constexpr long long kStageDrain = 1 << 20;

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

// Shared-memory layout of one stage: [3][TY + 2][TX + 8] velocity, then
// [TY + 2][TX + 8] viscosity, then (WB) [TY][TX] right-hand side, each
// starting on a 128-byte boundary; NS stages follow NS mbarriers.
template <int TX, int TY, bool WB = true>
struct Layout {
  static constexpr int PX = TX + 2 * kHX, PY = TY + 2;
  static constexpr int kU = 3 * PY * PX * 4, kE = PY * PX * 4, kB = WB ? TY * TX * 4 : 0;
  static constexpr int offE = round128(kU), offB = offE + round128(kE);
  static constexpr int stage = offB + round128(kB);
  static constexpr int tx_bytes = kU + kE + kB;  // the boxes' bytes, OOB fill included
  static __host__ __device__ constexpr int smem(int ns) { return 128 + ns * stage; }
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Block roles of one launch: per z chunk, ntx * nty tiles then nwall x-wall
// blocks.
struct SweepGrid {
  int tz, ntx, nty, nwall, nchunk;
  __host__ __device__ int per_chunk() const { return ntx * nty + nwall; }
  __host__ __device__ int blocks() const { return nchunk * per_chunk(); }
};

template <int TX, int TY>
inline SweepGrid sweep_grid(const Geom& g, int tz) {
  SweepGrid s;
  s.tz = tz;
  s.ntx = (g.n[0] + TX - 1) / TX;
  s.nty = (g.n[1] + TY - 1) / TY;
  s.nwall = (g.n[1] * tz + kWallRows - 1) / kWallRows;
  s.nchunk = (g.n[2] + tz - 1) / tz;
  return s;
}

// The block's role: chunk z0 / nz, and either an x-wall block (the row of
// its thread in the chunk, -1 past the last row) or the tile at (x0, y0).
struct Role {
  int z0, nz;
  bool wall;
  int row;
  int x0, y0;
};

__device__ __forceinline__ Role block_role(const Geom& g, const SweepGrid& sg, int TX, int TY) {
  Role r;
  const int chunk = blockIdx.x / sg.per_chunk();
  const int q = blockIdx.x - chunk * sg.per_chunk();
  r.z0 = chunk * sg.tz;
  r.nz = min(sg.tz, g.n[2] - r.z0);
  r.wall = q >= sg.ntx * sg.nty;
  r.row = -1;
  r.x0 = r.y0 = 0;
  if (r.wall) {
    const int row = (q - sg.ntx * sg.nty) * kWallRows + (int)threadIdx.x;
    if ((int)threadIdx.x < kWallRows && row < g.n[1] * r.nz) r.row = row;
  } else {
    r.x0 = (q % sg.ntx) * TX;
    r.y0 = (q / sg.ntx) * TY;
  }
  return r;
}

// The plane ring of one tile block.  plane(t, U, E, B) works on plane z0 + t,
// with U[d] and E[d] the staged velocity ([comp][y][x]) and viscosity
// ([y][x]) of plane z0 + t - 1 + d, and B the staged right-hand side of plane
// z0 + t (WB).  Returns false, after setting *err and draining, if a wait
// gave up; every thread of the block returns the same value.
template <int TX, int TY, int NS, bool WB, typename F>
__device__ __forceinline__ bool stream_planes(unsigned char* smem, const CUtensorMap* mu, const CUtensorMap* me,
                                              const CUtensorMap* mb, int bcomp, int x0, int y0, int z0, int nz,
                                              int* __restrict__ err, F plane) {
  using L = Layout<TX, TY, WB>;
  const int tid = threadIdx.x;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  const int np = nz + 2;  // planes z0 - 1 .. z0 + nz

  auto issue = [&](int q) {
    const int s = q % NS;
    const uint32_t bar = saddr(&bars[s]);
    const uint32_t base = saddr(stages + (size_t)s * L::stage);
    const int z = z0 - 1 + q;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(L::tx_bytes) : "memory");
    load_4d(base, mu, x0 - kHX, y0 - 1, z, 0, bar);
    load_3d(base + L::offE, me, x0 - kHX, y0 - 1, z, bar);
    if (WB) load_4d(base + L::offB, mb, x0, y0, z, bcomp, bar);
  };

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = 0; q < NS && q < np; ++q) issue(q);
  int issued = min(NS, np);  // planes whose loads were issued (the same in every thread)
  int landed = 0;            // planes 0 .. landed - 1 seen complete by this thread
  bool ok = true;
  for (int q = 0; q < 2 && ok; ++q)
    if (stage_wait(saddr(&bars[q % NS]), (uint32_t)((q / NS) & 1), kStageWait))
      landed = q + 1;
    else
      ok = false;

  for (int t = 0; t < nz; ++t) {
    if (ok) {
      if (stage_wait(saddr(&bars[(t + 2) % NS]), (uint32_t)(((t + 2) / NS) & 1), kStageWait))
        landed = t + 3;
      else
        ok = false;
    }
    if (ok) {
      const float* U[3];
      const float* E[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const unsigned char* st = stages + (size_t)((t + d) % NS) * L::stage;
        U[d] = reinterpret_cast<const float*>(st);
        E[d] = reinterpret_cast<const float*>(st + L::offE);
      }
      const float* B = reinterpret_cast<const float*>(stages + (size_t)((t + 1) % NS) * L::stage + L::offB);
      plane(t, U, E, B);
    }
    // plane k - 1's stage is free; every thread leaves together if one gave up
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    if (tid == 0 && t + NS < np) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(t + NS);
    }
    issued = min(t + 1 + NS, np);
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(err, 1);
      // no load may still be writing this block's shared memory when it exits
      for (int q = landed; q < issued; ++q) stage_wait(saddr(&bars[q % NS]), (uint32_t)((q / NS) & 1), kStageDrain);
    }
    __syncthreads();
  }
  return ok;
}

// The values of a staged neighbourhood: component q of the velocity and the
// viscosity at offset (dx, dy, dz) from the cell at (sx, sy) of the tile.
template <int TX, int TY>
struct Staged {
  const float* const* U;
  const float* const* E;
  int sx, sy;
  __device__ __forceinline__ float v(int q, int dx, int dy, int dz) const {
    constexpr int PX = TX + 2 * kHX, PY = TY + 2;
    return U[1 + dz][(q * PY + sy + dy) * PX + sx + dx];
  }
  __device__ __forceinline__ float e(int dx, int dy, int dz) const {
    constexpr int PX = TX + 2 * kHX;
    return E[1 + dz][(sy + dy) * PX + sx + dx];
  }
  // the faces below / above on every axis (unscaled cell sums, as CellEta)
  __device__ __forceinline__ void faces(float* elo, float* ehi) const {
    const float e0 = e(0, 0, 0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ox = a == 0, oy = a == 1, oz = a == 2;
      elo[a] = e(-ox, -oy, -oz) + e0;
      ehi[a] = e0 + e(ox, oy, oz);
    }
  }
  // u_c at the face neighbours and the cross-term values of component c, as
  // visc_gs_interior and tensor_interior gather them
  __device__ __forceinline__ void stencil(int c, float* ulo, float* uhi, float (*xa)[6]) const {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ox = a == 0, oy = a == 1, oz = a == 2;
      ulo[a] = v(c, -ox, -oy, -oz);
      uhi[a] = v(c, ox, oy, oz);
    }
    const int cx = c == 0, cy = c == 1, cz = c == 2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == c) continue;
      const int ax = a == 0, ay = a == 1, az = a == 2;
      xa[a][0] = v(a, cx, cy, cz);
      xa[a][1] = v(a, -cx, -cy, -cz);
      xa[a][2] = v(a, ax + cx, ay + cy, az + cz);
      xa[a][3] = v(a, ax - cx, ay - cy, az - cz);
      xa[a][4] = v(a, -ax + cx, -ay + cy, -az + cz);
      xa[a][5] = v(a, -ax - cx, -ay - cy, -az - cz);
    }
  }
};

// One colour sweep of component C.
template <int C, int TX, int TY, int NS>
__global__ void __launch_bounds__(kThreads) k_visc_smooth_tma(const __grid_constant__ CUtensorMap mu,
                                                              const __grid_constant__ CUtensorMap me,
                                                              const __grid_constant__ CUtensorMap mb,
                                                              float* __restrict__ u, const float* __restrict__ b,
                                                              const float* __restrict__ eta,
                                                              const __grid_constant__ Geom g, const SweepGrid sg,
                                                              int col, float beta, int hom, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const CellEta<float> ce{eta};
  const Role r = block_role(g, sg, TX, TY);
  if (r.wall) {
    if (r.row < 0) return;
    const int k = r.z0 + r.row / n1, j = r.row - (r.row / n1) * n1;
    int p[3] = {0, j, k};
    if (((j + k + col) & 1) == 0) visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
    p[0] = n0 - 1;
    if (n0 > 1 && ((n0 - 1 + j + k + col) & 1) == 0) visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
    return;
  }
  const float bs = beta * (g_ihh<float>(g) * float(CellEta<float>::kScale));
  constexpr int CPR = TX / 2;  // cells of one colour per tile row
  stream_planes<TX, TY, NS, true>(
      smem, &mu, &me, &mb, C, r.x0, r.y0, r.z0, r.nz, err,
      [&](int t, const float* const* U, const float* const* E, const float* B) {
        const int k = r.z0 + t;
#pragma unroll
        for (int rep = 0; rep < (TY * CPR + kThreads - 1) / kThreads; ++rep) {
          const int cell = (int)threadIdx.x + rep * kThreads;
          const int jr = cell / CPR, m = cell - jr * CPR;
          const int j = r.y0 + jr;
          const int i = r.x0 + 2 * m + ((j + k + col) & 1);
          if (jr >= TY || j >= n1 || i >= n0 - 1 || i == 0) continue;
          int p[3] = {i, j, k};
          if (j == 0 || j == n1 - 1 || k == 0 || k == n2 - 1) {
            visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
            continue;
          }
          const Staged<TX, TY> s{U, E, i - r.x0 + kHX, jr + 1};
          float elo[3], ehi[3], ulo[3], uhi[3], xa[3][6];
          s.faces(elo, ehi);
          s.stencil(C, ulo, uhi, xa);
          const float bc = B[jr * TX + (i - r.x0)];
          u[(size_t)C * g.ncell + cidx<3>(g, i, j, k)] = visc_gs_core<3, float>(C, elo, ehi, ulo, uhi, xa, bc, bs);
        }
      });
}

// out = u - beta L u, or b - (u - beta L u) when b != nullptr, for every cell
// and all three components (homogeneous walls when hom).
template <int TX, int TY, int NS>
__global__ void __launch_bounds__(kThreads) k_visc_op_tma(const __grid_constant__ CUtensorMap mu,
                                                          const __grid_constant__ CUtensorMap me,
                                                          const float* __restrict__ u, const float* __restrict__ b,
                                                          float* __restrict__ out, const float* __restrict__ eta,
                                                          const __grid_constant__ Geom g, const SweepGrid sg,
                                                          float beta, int hom, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const CellEta<float> ce{eta};
  const Role r = block_role(g, sg, TX, TY);
  if (r.wall) {
    if (r.row < 0) return;
    const int k = r.z0 + r.row / n1, j = r.row - (r.row / n1) * n1;
    int p[3] = {0, j, k};
    visc_op_cell<3, float, false>(u, b, out, ce, g, beta, hom, p, cidx<3>(g, 0, j, k));
    if (n0 > 1) {
      p[0] = n0 - 1;
      visc_op_cell<3, float, false>(u, b, out, ce, g, beta, hom, p, cidx<3>(g, n0 - 1, j, k));
    }
    return;
  }
  const float sc = g_ihh<float>(g) * float(CellEta<float>::kScale);
  stream_planes<TX, TY, NS, false>(
      smem, &mu, &me, nullptr, 0, r.x0, r.y0, r.z0, r.nz, err,
      [&](int t, const float* const* U, const float* const* E, const float*) {
        const int k = r.z0 + t;
#pragma unroll
        for (int rep = 0; rep < (TY * TX + kThreads - 1) / kThreads; ++rep) {
          const int cell = (int)threadIdx.x + rep * kThreads;
          const int jr = cell / TX, ii = cell - jr * TX;
          const int j = r.y0 + jr, i = r.x0 + ii;
          if (jr >= TY || j >= n1 || i >= n0 - 1 || i == 0) continue;
          int p[3] = {i, j, k};
          const int id = cidx<3>(g, i, j, k);
          if (j == 0 || j == n1 - 1 || k == 0 || k == n2 - 1) {
            visc_op_cell<3, float, false>(u, b, out, ce, g, beta, hom, p, id);
            continue;
          }
          const Staged<TX, TY> s{U, E, ii + kHX, jr + 1};
          float elo[3], ehi[3];
          s.faces(elo, ehi);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float ulo[3], uhi[3], xa[3][6];
            s.stencil(c, ulo, uhi, xa);
            const float u0 = s.v(c, 0, 0, 0);
            const float Lu = tensor_core<3, float>(c, u0, elo, ehi, ulo, uhi, xa, sc);
            const size_t o = (size_t)c * g.ncell + id;
            out[o] = op_out<float>(u0, Lu, beta, b, o);
          }
        }
      });
}

}  // namespace tma
}  // namespace hb
