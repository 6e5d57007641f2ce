// Kernels of the learned initial-guess network (U-Net on the nodal grid).
//
// Activations are channels-last BF16: element (point p, channel c) at
// p*C + c, points x fastest on a padded box of X*Y*Z points.  Convolutions
// are implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16 inputs,
// FP32 accumulation): rows = 16 points, columns = 8 output channels,
// k = 16 input channels of one of the 3^D taps.  Taps are the offsets in
// {-1,0,1}^D in lexicographic order (x slowest), zero padding outside.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace hb {
namespace nn {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int D>
__device__ __forceinline__ void tap_offset(int t, int* o) {
  if (D == 3) {
    o[0] = t / 9 - 1;
    o[1] = (t / 3) % 3 - 1;
    o[2] = t % 3 - 1;
  } else {
    o[0] = t / 3 - 1;
    o[1] = t % 3 - 1;
    o[2] = 0;
  }
}

struct Box {
  int X, Y, Z;
};

// point index of p shifted by o, or -1 outside the box
__device__ __forceinline__ long long shifted(const Box& b, int i, int j, int k, const int* o) {
  int a = i + o[0], c = j + o[1], e = k + o[2];
  if (a < 0 || a >= b.X || c < 0 || c >= b.Y || e < 0 || e >= b.Z) return -1;
  return (long long)a + (long long)b.X * ((long long)c + (long long)b.Y * e);
}

__device__ __forceinline__ void coords(const Box& b, long long p, int& i, int& j, int& k) {
  i = (int)(p % b.X);
  long long r = p / b.X;
  j = (int)(r % b.Y);
  k = (int)(r / b.Y);
}

// out[p, out_off + co] = act(bias[co] + sum_tap sum_ci in[p + o_tap, ci] W[tap, co, ci])
// for the NTB*8 output channels of slice blockIdx.y.  4 warps, 16 points each.
// W: [taps][Cout][Cin] BF16 (Cin multiple of 16).  bias may be null.
template <int D, int NTB>
__global__ void __launch_bounds__(128) k_conv_fwd(const bf16* __restrict__ in, int Cin, const bf16* __restrict__ W,
                                                  const float* __restrict__ bias, int Cout, bf16* __restrict__ out,
                                                  int out_stride, int out_off, int relu, Box box) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const long long P = (long long)box.X * box.Y * box.Z;
  const long long p0 = ((long long)blockIdx.x * 4 + warp) * 16;
  if (p0 >= P) return;
  const int co_base = blockIdx.y * NTB * 8;
  long long pr[2] = {p0 + g, p0 + g + 8};
  int ci[2], cj[2], ck[2];
  bool valid[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    valid[r] = pr[r] < P;
    coords(box, valid[r] ? pr[r] : 0, ci[r], cj[r], ck[r]);
  }
  float acc[NTB][4];
#pragma unroll
  for (int n = 0; n < NTB; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const int T = D == 3 ? 27 : 9;
  const int KC = Cin / 16;
  for (int tap = 0; tap < T; ++tap) {
    int o[3];
    tap_offset<D>(tap, o);
    long long q[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) q[r] = valid[r] ? shifted(box, ci[r], cj[r], ck[r], o) : -1;
    for (int kc = 0; kc < KC; ++kc) {
      uint32_t A[4];
      const int cb = kc * 16 + 2 * t4;
      A[0] = q[0] >= 0 ? ld32(in + q[0] * Cin + cb) : 0u;
      A[1] = q[1] >= 0 ? ld32(in + q[1] * Cin + cb) : 0u;
      A[2] = q[0] >= 0 ? ld32(in + q[0] * Cin + cb + 8) : 0u;
      A[3] = q[1] >= 0 ? ld32(in + q[1] * Cin + cb + 8) : 0u;
#pragma unroll
      for (int n = 0; n < NTB; ++n) {
        const bf16* wp = W + ((size_t)tap * Cout + co_base + n * 8 + g) * Cin + cb;
        mma_bf16(acc[n], A, ld32(wp), ld32(wp + 8));
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NTB; ++n) {
    const int co = co_base + n * 8 + 2 * t4;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!valid[r]) continue;
      float v0 = acc[n][2 * r] + b0, v1 = acc[n][2 * r + 1] + b1;
      if (relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      *reinterpret_cast<uint32_t*>(out + pr[r] * out_stride + out_off + co) =
          pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
    }
  }
}

// gW[tap, co, ci] += sum_p gz[p, co] x[p + o_tap, ci] over one chunk of points.
// blockIdx.x*4 + warp selects a (16 co) x (8 ci) tile, blockIdx.y the tap,
// blockIdx.z the chunk.  FP32 atomics into gW.
template <int D>
__global__ void __launch_bounds__(128) k_conv_wgrad(const bf16* __restrict__ x, int Cin, const bf16* __restrict__ gz,
                                                    int Cout, float* __restrict__ gW, Box box, int chunk) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int nci = Cin / 8, nco = Cout / 16;
  const int pair = blockIdx.x * 4 + warp;
  if (pair >= nci * nco) return;
  const int co0 = (pair / nci) * 16, ci0 = (pair % nci) * 8;
  const int tap = blockIdx.y;
  int o[3];
  tap_offset<D>(tap, o);
  const long long P = (long long)box.X * box.Y * box.Z;
  const long long pb = (long long)blockIdx.z * chunk;
  const long long pe = pb + chunk < P ? pb + chunk : P;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const bf16 zero = __float2bfloat16_rn(0.f);
  for (long long p0 = pb; p0 < pe; p0 += 16) {
    // A (16 co x 16 points): a(row co, col p) = gz[p, co]
    bf16 av[8];
    const int kcol[4] = {2 * t4, 2 * t4 + 1, 2 * t4 + 8, 2 * t4 + 9};
    long long pk[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) pk[s] = p0 + kcol[s];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const bool ok = pk[s] < pe;
      av[2 * s] = ok ? gz[pk[s] * Cout + co0 + g] : zero;      // row g
      av[2 * s + 1] = ok ? gz[pk[s] * Cout + co0 + g + 8] : zero;  // row g + 8
    }
    uint32_t A[4];
    A[0] = pack2(av[0], av[2]);  // row g, k = 2t, 2t+1
    A[1] = pack2(av[1], av[3]);  // row g+8
    A[2] = pack2(av[4], av[6]);  // row g, k = 2t+8, 2t+9
    A[3] = pack2(av[5], av[7]);  // row g+8
    // B (16 points x 8 ci): b(row p, col ci) = x[p + o, ci]
    bf16 bv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      bv[s] = zero;
      if (pk[s] < pe) {
        int i, j, k;
        coords(box, pk[s], i, j, k);
        long long q = shifted(box, i, j, k, o);
        if (q >= 0) bv[s] = x[q * Cin + ci0 + g];
      }
    }
    mma_bf16(acc, A, pack2(bv[0], bv[1]), pack2(bv[2], bv[3]));
  }
  float* base = gW + ((size_t)tap * Cout + co0) * Cin + ci0;
  atomicAdd(base + (size_t)g * Cin + 2 * t4, acc[0]);
  atomicAdd(base + (size_t)g * Cin + 2 * t4 + 1, acc[1]);
  atomicAdd(base + (size_t)(g + 8) * Cin + 2 * t4, acc[2]);
  atomicAdd(base + (size_t)(g + 8) * Cin + 2 * t4 + 1, acc[3]);
}

}  // namespace nn
}  // namespace hb
