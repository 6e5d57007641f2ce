// The U-Net convolution on the 5th-generation tensor cores (tcgen05): an
// implicit GEMM D[p, co] = sum_tap sum_ci X[p + o_tap, ci] W[tap, co, ci]
// with M = 128 points per CTA, N = Cout, K = Cin per tap.  Per tap the CTA
// gathers its 128 shifted input rows and the tap's Cout x Cin weights into
// shared memory (K-major, no swizzle: core matrices of 8 rows x 16 bytes),
// one thread issues Cin/16 tcgen05.mma (BF16 in, FP32 accumulate in TMEM),
// tcgen05.commit arrives on an mbarrier that the CTA waits on (bounded)
// before the next tap overwrites the operands; the epilogue reads the
// accumulators with tcgen05.ld (warp w owns TMEM lanes 32w .. 32w+31, i.e.
// its 32 points), adds the bias, applies ReLU and stores BF16.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

#include "hb_unet_kernels.cuh"

namespace hb {
namespace nn {

constexpr int kTcM = 128;                 // points per CTA (the MMA's M)
// mbarrier polls before a wait on the tensor cores gives up.  A CTA that
// gives up sets the network's error flag (the host then reports
// HBF_ERR_TIMEOUT and discards every output of that forward pass), waits
// again on the same phase for up to kTcDrainLimit polls so that no MMA it
// issued is still writing its TMEM columns or reading its shared memory, and
// only then frees its TMEM and exits.  Completion of one CTA's MMAs takes
// microseconds, so neither limit is reached in normal operation.
constexpr long long kTcWaitLimit = 1 << 24;
constexpr long long kTcDrainLimit = 1 << 27;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for a K-major operand without swizzling:
// start address, byte stride between core matrices along K (leading) and
// along M/N (stride), descriptor version 1; base offset 0, layout 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM columns for an accumulator of n FP32 columns (a power of two >= 32)
__host__ __device__ constexpr int tc_cols(int n) {
  return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}

__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity,
                                                 long long limit = kTcWaitLimit) {
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

// dynamic shared memory of one CTA: the A and B tiles, plus slack so that
// descriptor strides read in either order stay inside the allocation
constexpr int kTcSlack = 16384;
__host__ __device__ constexpr int tc_smem_bytes(int cin, int cout) { return (kTcM + cout) * cin * 2 + kTcSlack; }

// out[p, out_off + co] = act(bias[co] + sum_tap sum_ci in[p + o_tap, ci] W[tap, co, ci]).
// Requires Cin % 16 == 0, Cout % 16 == 0, 16 <= Cout <= 256; tcols = tc_cols(Cout).
// *err is set when a wait on the tensor cores gives up (the outputs of that
// CTA are then not written).
template <int D>
__global__ void __launch_bounds__(kTcM, 1) k_conv_fwd_tc(const bf16* __restrict__ in, int Cin,
                                                        const bf16* __restrict__ W, const float* __restrict__ bias,
                                                        int Cout, bf16* __restrict__ out, int out_stride,
                                                        int out_off, int relu, Box box, int tcols,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  unsigned char* sA = smem;                             // kTcM rows x Cin
  unsigned char* sB = smem + (size_t)kTcM * Cin * 2;    // Cout rows x Cin
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KC = Cin / 8;  // 16-byte chunks per row
  const long long P = (long long)box.X * box.Y * box.Z;
  const long long p = (long long)blockIdx.x * kTcM + tid;
  const bool valid = p < P;
  int ci = 0, cj = 0, ck = 0;
  if (valid) coords(box, p, ci, cj, ck);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t bar = smem_u32(&mbar);
  const uint32_t idesc = tc_idesc(kTcM, Cout);
  const uint32_t sbo = (uint32_t)KC * 128u;  // next 8-row group
  const int T = D == 3 ? 27 : 9;
  bool ok = true;
  uint32_t parity = 0;
  for (int tap = 0; tap < T && ok; ++tap) {  // ok is the same in every thread
    int o[3];
    tap_offset<D>(tap, o);
    const long long q = valid ? shifted(box, ci, cj, ck, o) : -1;
    // this thread's row of A: the shifted point's channels (zero outside)
    unsigned char* arow = sA + (size_t)((tid >> 3) * KC) * 128 + (tid & 7) * 16;
    for (int k8 = 0; k8 < KC; ++k8) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q >= 0) v = *reinterpret_cast<const uint4*>(in + q * Cin + 8 * k8);
      *reinterpret_cast<uint4*>(arow + (size_t)k8 * 128) = v;
    }
    // the tap's weights, Cout rows of Cin
    const bf16* Wt = W + (size_t)tap * Cout * Cin;
    for (int idx = tid; idx < Cout * KC; idx += kTcM) {
      const int r = idx / KC, k8 = idx - r * KC;
      const uint4 v = *reinterpret_cast<const uint4*>(Wt + (size_t)r * Cin + 8 * k8);
      *reinterpret_cast<uint4*>(sB + (size_t)((r >> 3) * KC + k8) * 128 + (r & 7) * 16) = v;
    }
    // make the generic-proxy stores visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int kc = 0; kc < Cin / 16; ++kc) {
        const uint64_t ad = tc_desc(smem_u32(sA) + (uint32_t)kc * 256u, 128u, sbo);
        const uint64_t bd = tc_desc(smem_u32(sB) + (uint32_t)kc * 256u, 128u, sbo);
        const uint32_t acc = (tap > 0 || kc > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
    // every thread waits for the MMAs before the operands are overwritten;
    // the block agrees on the outcome so that all threads leave together
    const bool mine = mbar_wait_parity(bar, parity);
    ok = __syncthreads_and(mine ? 1 : 0) != 0;
    if (ok) parity ^= 1u;  // on failure parity keeps the phase still pending
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < Cout; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_base + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (valid) {
        uint32_t packed[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          float v0 = __uint_as_float(r[2 * m]) + (bias ? bias[c0 + 2 * m] : 0.f);
          float v1 = __uint_as_float(r[2 * m + 1]) + (bias ? bias[c0 + 2 * m + 1] : 0.f);
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          packed[m] = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
        }
        uint4* dst = reinterpret_cast<uint4*>(out + p * out_stride + out_off + c0);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // drain: the MMAs of the pending phase must finish before TMEM is freed
    mbar_wait_parity(bar, parity, kTcDrainLimit);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
}

// ---------------------------------------------------------------------------
// Halo variant for the layers whose whole tap set fits in shared memory.  The
// CTA's 128 points are an 8 (x) x 16 (y) tile of one z plane.  Its input halo
// (10 x 18 x 3 points in 3D, 10 x 18 in 2D, zero outside the box) is staged
// once, one plane of 16-byte channel chunks per K chunk, rows at a 16-byte
// stride; then the operand of tap (dx, dy, dz) is a descriptor into that halo:
// 8 consecutive halo rows (one tile row shifted by dx) form a core matrix at
// any start row, the next tile row is 10 halo rows further (SBO = 160 bytes)
// and the next K chunk one plane further (LBO).  The weights of all taps are
// staged once as well, so one thread issues all 3^d * Cin/16 MMAs back to back
// and the CTA waits once.
// ---------------------------------------------------------------------------
constexpr int kHaloX = 10, kHaloY = 18;
constexpr int kTcHaloMaxSmem = 200 * 1024;  // dynamic shared memory the halo variant may use

__host__ __device__ constexpr int tc_halo_rows(int d) { return kHaloX * kHaloY * (d == 3 ? 3 : 1); }

__host__ __device__ constexpr int tc_halo_smem_bytes(int d, int cin, int cout) {
  return tc_halo_rows(d) * cin * 2 + (d == 3 ? 27 : 9) * cout * cin * 2 + kTcSlack;
}

template <int D>
__global__ void __launch_bounds__(kTcM, 1) k_conv_fwd_tc_halo(const bf16* __restrict__ in, int Cin,
                                                             const bf16* __restrict__ W,
                                                             const float* __restrict__ bias, int Cout,
                                                             bf16* __restrict__ out, int out_stride, int out_off,
                                                             int relu, Box box, int tcols, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  constexpr int T = D == 3 ? 27 : 9;
  constexpr int HR = tc_halo_rows(D);
  const int KC = Cin / 8;
  const uint32_t plane = (uint32_t)HR * 16u;            // one 16-byte channel chunk of every halo row
  unsigned char* sH = smem;                              // KC planes
  unsigned char* sB = smem + (size_t)KC * plane;         // T taps x Cout rows x Cin
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntx = box.X / 8, nty = (box.Y + 15) / 16;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty;
  const int z = t / nty;
  const int x0 = tx * 8, y0 = ty * 16;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // input halo, zero outside the box
  for (int idx = tid; idx < HR * KC; idx += kTcM) {
    const int h = idx / KC, k8 = idx - h * KC;
    const int xx = h % kHaloX, r = h / kHaloX, yy = r % kHaloY, zz = r / kHaloY;
    const int gx = x0 - 1 + xx, gy = y0 - 1 + yy, gz = D == 3 ? z - 1 + zz : 0;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gx >= 0 && gx < box.X && gy >= 0 && gy < box.Y && gz >= 0 && gz < box.Z) {
      const long long q = (long long)gx + (long long)box.X * ((long long)gy + (long long)box.Y * gz);
      v = *reinterpret_cast<const uint4*>(in + q * Cin + 8 * k8);
    }
    *reinterpret_cast<uint4*>(sH + (size_t)k8 * plane + (size_t)h * 16) = v;
  }
  // weights of every tap, core-matrix layout per tap
  for (int idx = tid; idx < T * Cout * KC; idx += kTcM) {
    const int k8 = idx % KC, rr = idx / KC;  // rr = tap * Cout + row
    const int tap = rr / Cout, r = rr - tap * Cout;
    const uint4 v = *reinterpret_cast<const uint4*>(W + (size_t)rr * Cin + 8 * k8);
    *reinterpret_cast<uint4*>(sB + (size_t)tap * Cout * Cin * 2 + (size_t)((r >> 3) * KC + k8) * 128 +
                              (r & 7) * 16) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t bar = smem_u32(&mbar);
  if (tid == 0) {
    const uint32_t idesc = tc_idesc(kTcM, Cout);
    const uint32_t hbase = smem_u32(sH), bbase = smem_u32(sB);
    for (int tap = 0; tap < T; ++tap) {
      int o[3];
      tap_offset<D>(tap, o);
      const int row0 = ((D == 3 ? (1 + o[2]) * kHaloY : 0) + (1 + o[1])) * kHaloX + (1 + o[0]);
      for (int kc = 0; kc < Cin / 16; ++kc) {
        const uint64_t ad = tc_desc(hbase + (uint32_t)(2 * kc) * plane + (uint32_t)row0 * 16u, plane,
                                    (uint32_t)kHaloX * 16u);
        const uint64_t bd = tc_desc(bbase + (uint32_t)tap * Cout * Cin * 2 + (uint32_t)kc * 256u, 128u,
                                    (uint32_t)KC * 128u);
        const uint32_t acc = (tap > 0 || kc > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
  }
  const bool ok = __syncthreads_and(mbar_wait_parity(bar, 0u) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // row tid of D is the tile point (x0 + tid % 8, y0 + tid / 8, z)
  const int px = x0 + (tid & 7), py = y0 + (tid >> 3);
  const bool valid = py < box.Y;
  const long long p = (long long)px + (long long)box.X * ((long long)py + (long long)box.Y * (D == 3 ? z : 0));
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < Cout; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_base + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (valid) {
        uint32_t packed[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          float v0 = __uint_as_float(r[2 * m]) + (bias ? bias[c0 + 2 * m] : 0.f);
          float v1 = __uint_as_float(r[2 * m + 1]) + (bias ? bias[c0 + 2 * m + 1] : 0.f);
          if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          }
          packed[m] = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
        }
        uint4* dst = reinterpret_cast<uint4*>(out + p * out_stride + out_off + c0);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
      }
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait_parity(bar, 0u, kTcDrainLimit);  // drain before TMEM is freed
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcols) : "memory");
}

}  // namespace nn
}  // namespace hb
