// The finest-level FP32 red-black Gauss-Seidel sweep of one velocity
// component and one colour (Eq. 16, face viscosities formed from the cell
// viscosity), with its operands staged in shared memory by the tensor memory
// accelerator (3D only).
//
// A block owns a tile of TX x TY cells in x, y and a chunk of TZ planes in z,
// and streams the planes z0 - 1 .. z0 + TZ through a ring of NS stages: one
// thread issues, per plane, three cp.async.bulk.tensor loads (the three
// velocity components and the cell viscosity over the tile with a halo of
// kHX cells in x and one row in y, and the right-hand side of the component
// over the tile) that complete on the stage's mbarrier, while the block
// updates the plane two stages behind from shared memory.  A load's x
// coordinate is a multiple of 4 floats (16 bytes): the x halo is 4 cells so
// that x0 - 4 stays aligned.  Coordinates outside the grid read zeros, which
// only cells that take the global path below would see.
//
// Within a sweep of one colour, every value the update reads (u_c of the
// other colour, the other components, eta, b) is left unchanged by the
// sweep, so stale or fresh copies are the same and the staged planes never
// need refreshing.  The update of an interior cell is visc_gs_core on the
// same gathered values as visc_gs_interior: the results are the same bit for
// bit as those of k_visc_smooth_c.  Cells on a y or z wall take the global
// path (visc_smooth_cell) inside the tile; the cells on the two x walls,
// whose warps would otherwise run the wall stencil next to interior cells,
// are taken by kWallRows-row wall blocks placed after the tiles of each z
// chunk, so that they run while that chunk's planes are still in L2.
//
// Every mbarrier wait is bounded (kStageWait polls).  A block that gives up
// sets *err, stops updating, waits (bounded again) for the loads it has in
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
// [TY + 2][TX + 8] viscosity, then [TY][TX] right-hand side, each starting on
// a 128-byte boundary; NS stages follow NS mbarriers.
template <int TX, int TY>
struct Layout {
  static constexpr int PX = TX + 2 * kHX, PY = TY + 2;
  static constexpr int kU = 3 * PY * PX * 4, kE = PY * PX * 4, kB = TY * TX * 4;
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

template <int C, int TX, int TY, int NS>
__global__ void __launch_bounds__(kThreads) k_visc_smooth_tma(const __grid_constant__ CUtensorMap mu,
                                                              const __grid_constant__ CUtensorMap me,
                                                              const __grid_constant__ CUtensorMap mb,
                                                              float* __restrict__ u, const float* __restrict__ b,
                                                              const float* __restrict__ eta,
                                                              const __grid_constant__ Geom g, const SweepGrid sg,
                                                              int col, float beta, int hom, int* __restrict__ err) {
  using L = Layout<TX, TY>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int chunk = blockIdx.x / sg.per_chunk();
  const int r = blockIdx.x - chunk * sg.per_chunk();
  const int z0 = chunk * sg.tz;
  const int nz = min(sg.tz, n2 - z0);
  const CellEta<float> ce{eta};

  if (r >= sg.ntx * sg.nty) {
    // x-wall block: one thread per row (j, k) of this chunk
    const int row = (r - sg.ntx * sg.nty) * kWallRows + tid;
    if (tid >= kWallRows || row >= n1 * nz) return;
    const int k = z0 + row / n1, j = row - (row / n1) * n1;
    int p[3] = {0, j, k};
    if (((j + k + col) & 1) == 0) visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
    p[0] = n0 - 1;
    if (n0 > 1 && ((n0 - 1 + j + k + col) & 1) == 0) visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
    return;
  }

  const int tx = r % sg.ntx, ty = r / sg.ntx;
  const int x0 = tx * TX, y0 = ty * TY;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  const int np = nz + 2;  // planes z0 - 1 .. z0 + nz

  auto issue = [&](int q) {
    const int s = q % NS;
    const uint32_t bar = saddr(&bars[s]);
    const uint32_t base = saddr(stages + (size_t)s * L::stage);
    const int z = z0 - 1 + q;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(L::tx_bytes) : "memory");
    load_4d(base, &mu, x0 - kHX, y0 - 1, z, 0, bar);
    load_3d(base + L::offE, &me, x0 - kHX, y0 - 1, z, bar);
    load_4d(base + L::offB, &mb, x0, y0, z, C, bar);
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

  const float bs = beta * (g_ihh<float>(g) * float(CellEta<float>::kScale));
  constexpr int PX = L::PX;
  constexpr int CPR = TX / 2;  // cells of one colour per tile row
  for (int t = 0; t < nz; ++t) {
    if (ok) {
      if (stage_wait(saddr(&bars[(t + 2) % NS]), (uint32_t)(((t + 2) / NS) & 1), kStageWait))
        landed = t + 3;
      else
        ok = false;
    }
    const int k = z0 + t;
    const float* U[3];  // planes k - 1, k, k + 1: [comp][y][x]
    const float* E[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const unsigned char* st = stages + (size_t)((t + d) % NS) * L::stage;
      U[d] = reinterpret_cast<const float*>(st);
      E[d] = reinterpret_cast<const float*>(st + L::offE);
    }
    const float* B = reinterpret_cast<const float*>(stages + (size_t)((t + 1) % NS) * L::stage + L::offB);
    if (ok) {
#pragma unroll
      for (int rep = 0; rep < (TY * CPR + kThreads - 1) / kThreads; ++rep) {
        const int cell = tid + rep * kThreads;
        const int jr = cell / CPR, m = cell - jr * CPR;
        const int j = y0 + jr;
        const int i = x0 + 2 * m + ((j + k + col) & 1);
        if (jr >= TY || j >= n1 || i >= n0 - 1 || i == 0) continue;
        int p[3] = {i, j, k};
        if (j == 0 || j == n1 - 1 || k == 0 || k == n2 - 1) {
          visc_smooth_cell<3, float, C, false>(u, b, ce, g, beta, hom, p);
          continue;
        }
        const int sx = i - x0 + kHX, sy = jr + 1;
        // value of component q at offset (dx, dy, dz) from the cell
        auto V = [&](int q, int dx, int dy, int dz) -> float {
          return U[1 + dz][(q * L::PY + sy + dy) * PX + sx + dx];
        };
        auto W = [&](int dx, int dy, int dz) -> float { return E[1 + dz][(sy + dy) * PX + sx + dx]; };
        const float e0 = W(0, 0, 0);
        float elo[3], ehi[3], ulo[3], uhi[3], xa[3][6];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int ox = a == 0, oy = a == 1, oz = a == 2;
          elo[a] = W(-ox, -oy, -oz) + e0;
          ehi[a] = e0 + W(ox, oy, oz);
          ulo[a] = V(C, -ox, -oy, -oz);
          uhi[a] = V(C, ox, oy, oz);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a == C) continue;
          const int cx = C == 0, cy = C == 1, cz = C == 2;
          const int ax = a == 0, ay = a == 1, az = a == 2;
          xa[a][0] = V(a, cx, cy, cz);
          xa[a][1] = V(a, -cx, -cy, -cz);
          xa[a][2] = V(a, ax + cx, ay + cy, az + cz);
          xa[a][3] = V(a, ax - cx, ay - cy, az - cz);
          xa[a][4] = V(a, -ax + cx, -ay + cy, -az + cz);
          xa[a][5] = V(a, -ax - cx, -ay - cy, -az - cz);
        }
        const float bc = B[jr * TX + (i - x0)];
        u[(size_t)C * g.ncell + cidx<3>(g, i, j, k)] = visc_gs_core<3, float>(C, elo, ehi, ulo, uhi, xa, bc, bs);
      }
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
}

}  // namespace tma
}  // namespace hb
