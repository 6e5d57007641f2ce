// The learned initial guess: a 4-level U-Net (16-32-64-128 channels, 3^D
// convolutions, ReLU, 2^D average pooling, nearest upsampling with skip
// concatenation, 1x1 head) evaluated and trained by this library's own
// kernels: BF16 tensor-core convolutions with FP32 accumulation
// (hb_unet_kernels.cuh), FP32 master weights and Adam.
//
// The network maps the normalised warm-start residual of the nodal projection
// solve (Eq. 17) to a correction of its initial guess; the multigrid solve
// remains the judge and runs to the same tolerance from that guess.
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "hb_internal.h"
#include "hb_unet_kernels.cuh"
#include "hb_unet_tc.cuh"

using hb::nn::bf16;
using hb::nn::Box;

namespace hb {
namespace nn {

constexpr int kCh[4] = {16, 32, 64, 128};

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
__global__ void k_f32_to_bf16(bf16* __restrict__ o, const float* __restrict__ i, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    o[t] = __float2bfloat16_rn(i[t]);
}

// input x (P points, one value) -> channel 0 of a 16-channel BF16 tensor (others 0)
__global__ void k_pack_input(bf16* __restrict__ o, const float* __restrict__ x, long long P) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P * 16; t += (long long)gridDim.x * blockDim.x)
    o[t] = __float2bfloat16_rn((t & 15) == 0 ? x[t >> 4] : 0.f);
}

// 2^D average of children into the parent (channels-last)
template <int D>
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int C, Box fine) {
  const Box c{fine.X / 2, fine.Y / 2, D == 3 ? fine.Z / 2 : 1};
  const long long n = (long long)c.X * c.Y * c.Z * C;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % C);
    long long P = t / C;
    int I, J, K;
    coords(c, P, I, J, K);
    // x first, then y, then z (pairwise means, as the reference)
    float vz[2];
    for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk) {
      float vy[2];
      for (int jj = 0; jj < 2; ++jj) {
        long long q0 = (long long)(2 * I) + (long long)fine.X * ((long long)(2 * J + jj) + (long long)fine.Y * (D == 3 ? 2 * K + kk : 0));
        vy[jj] = 0.5f * (__bfloat162float(in[q0 * C + ch]) + __bfloat162float(in[(q0 + 1) * C + ch]));
      }
      vz[kk] = 0.5f * (vy[0] + vy[1]);
    }
    const float v = D == 3 ? 0.5f * (vz[0] + vz[1]) : vz[0];
    out[t] = __float2bfloat16_rn(v);
  }
}

// nearest upsampling of in (coarse, Cin channels) into channels [0, Cin) of out (stride Cs)
template <int D>
__global__ void k_upsample(const bf16* __restrict__ in, int Cin, bf16* __restrict__ out, int Cs, Box fine) {
  const Box c{fine.X / 2, fine.Y / 2, D == 3 ? fine.Z / 2 : 1};
  const long long n = (long long)fine.X * fine.Y * fine.Z * Cin;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % Cin);
    long long p = t / Cin;
    int i, j, k;
    coords(fine, p, i, j, k);
    long long P = (long long)(i / 2) + (long long)c.X * ((long long)(j / 2) + (long long)c.Y * (k / 2));
    out[p * Cs + ch] = in[P * Cin + ch];
  }
}

// copy C channels of src (stride C) into channels [off, off+C) of dst (stride Cs)
__global__ void k_copy_channels(const bf16* __restrict__ src, int C, bf16* __restrict__ dst, int Cs, int off, long long P) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P * C; t += (long long)gridDim.x * blockDim.x)
    dst[(t / C) * Cs + off + t % C] = src[t];
}

// head: y[p] = sum_c h[p, c] w[c] + b (FP32 output)
__global__ void k_head_fwd(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                           float* __restrict__ y, long long P) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    float acc = b[0];
    for (int c = 0; c < 16; ++c) acc += __bfloat162float(h[p * 16 + c]) * w[c];
    y[p] = acc;
  }
}

// head backward: gh[p, c] = gy[p] w[c] (BF16); gw[c] += sum gy h[:, c]; gb += sum gy
__global__ void k_head_bwd(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ gy,
                           bf16* __restrict__ gh, float* __restrict__ gw, float* __restrict__ gb, long long P) {
  float aw[16];
  float ab = 0.f;
  for (int c = 0; c < 16; ++c) aw[c] = 0.f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const float g = gy[p];
    ab += g;
    for (int c = 0; c < 16; ++c) {
      aw[c] += g * __bfloat162float(h[p * 16 + c]);
      gh[p * 16 + c] = __float2bfloat16_rn(g * w[c]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    ab += __shfl_xor_sync(0xffffffffu, ab, off);
    for (int c = 0; c < 16; ++c) aw[c] += __shfl_xor_sync(0xffffffffu, aw[c], off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(gb, ab);
    for (int c = 0; c < 16; ++c) atomicAdd(gw + c, aw[c]);
  }
}

// ReLU backward in place: g *= (y > 0)
__global__ void k_relu_bwd(bf16* __restrict__ g, const bf16* __restrict__ y, long long n) {
  const bf16 z = __float2bfloat16_rn(0.f);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[t]) > 0.f)) g[t] = z;
}

// bias gradient: gb[c] += sum_p g[p, c]
__global__ void k_bias_grad(const bf16* __restrict__ g, int C, long long P, float* __restrict__ gb) {
  extern __shared__ float sh[];
  const int c = threadIdx.x % C;
  const int rows = blockDim.x / C;
  const int r = threadIdx.x / C;
  float acc = 0.f;
  if (r < rows)
    for (long long p = (long long)blockIdx.x * rows + r; p < P; p += (long long)gridDim.x * rows)
      acc += __bfloat162float(g[p * C + c]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < C) {
    float s = 0.f;
    for (int q = 0; q < rows; ++q) s += sh[q * C + threadIdx.x];
    atomicAdd(gb + threadIdx.x, s);
  }
}

// upsample backward: g_coarse[P, c] = sum over children of g_cat[child, c] (c < Cup)
template <int D>
__global__ void k_upsample_bwd(const bf16* __restrict__ gcat, int Cs, int Cup, bf16* __restrict__ gc, Box fine) {
  const Box c{fine.X / 2, fine.Y / 2, D == 3 ? fine.Z / 2 : 1};
  const long long n = (long long)c.X * c.Y * c.Z * Cup;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % Cup);
    long long P = t / Cup;
    int I, J, K;
    coords(c, P, I, J, K);
    float vz[2];
    for (int kk = 0; kk < (D == 3 ? 2 : 1); ++kk) {
      float vy[2];
      for (int jj = 0; jj < 2; ++jj) {
        long long q0 = (long long)(2 * I) + (long long)fine.X * ((long long)(2 * J + jj) + (long long)fine.Y * (D == 3 ? 2 * K + kk : 0));
        vy[jj] = __bfloat162float(gcat[q0 * Cs + ch]) + __bfloat162float(gcat[(q0 + 1) * Cs + ch]);
      }
      vz[kk] = vy[0] + vy[1];
    }
    gc[t] = __float2bfloat16_rn(D == 3 ? vz[0] + vz[1] : vz[0]);
  }
}

// gradient of an encoder output: pool backward of g_next (coarse) plus the
// skip part of the decoder's concatenation gradient
template <int D>
__global__ void k_pool_bwd_add(const bf16* __restrict__ gnext, const bf16* __restrict__ gcat, int Cs, int off,
                               bf16* __restrict__ gout, int C, Box fine) {
  const Box c{fine.X / 2, fine.Y / 2, D == 3 ? fine.Z / 2 : 1};
  const float w = D == 3 ? 0.125f : 0.25f;
  const long long n = (long long)fine.X * fine.Y * fine.Z * C;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(t % C);
    long long p = t / C;
    int i, j, k;
    coords(fine, p, i, j, k);
    long long P = (long long)(i / 2) + (long long)c.X * ((long long)(j / 2) + (long long)c.Y * (k / 2));
    const float pooled = __bfloat162float(__float2bfloat16_rn(__bfloat162float(gnext[P * C + ch]) * w));
    gout[t] = __float2bfloat16_rn(pooled + __bfloat162float(gcat[p * Cs + off + ch]));
  }
}

// transposed, flipped weights for the input gradient:
// Wt[tap', ci, co] = W[tap, co, ci], tap' = mirror of tap
template <int D>
__global__ void k_flip_transpose(const bf16* __restrict__ W, bf16* __restrict__ Wt, int Cout, int Cin) {
  const int T = D == 3 ? 27 : 9;
  const long long n = (long long)T * Cout * Cin;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(t % Cin);
    const int co = (int)((t / Cin) % Cout);
    const int tap = (int)(t / ((long long)Cin * Cout));
    Wt[((size_t)(T - 1 - tap) * Cin + ci) * Cout + co] = W[t];
  }
}

// MSE over masked points: gy = 2 mask (y - t) / nvalid; partial sums of the loss
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask,
                      float* __restrict__ gy, double* __restrict__ part, long long P, double inv_n) {
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    const double r = (double)mask[p] * ((double)y[p] - (double)t[p]);
    acc += r * r;
    gy[p] = (float)(2.0 * r * inv_n);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s * inv_n;
  }
}

// per-block sums of a 0/1 mask
__global__ void k_mask_sum(const float* __restrict__ mask, double* __restrict__ part, long long P) {
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x)
    acc += (double)mask[p];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// Adam on FP32 master weights; refreshes the BF16 copy and clears the gradient
__global__ void k_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ wb, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    const float ww = w[t] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w[t] = ww;
    if (wb) wb[t] = __float2bfloat16_rn(ww);
    g[t] = 0.f;
  }
}

}  // namespace nn
}  // namespace hb

// ---------------------------------------------------------------------------
// the network
// ---------------------------------------------------------------------------
struct hbf_unet {
  int d = 2;
  bool train = false;
  cudaStream_t stream = nullptr;
  hb::nn::Box box[4];
  long long P[4];
  struct Layer {
    int cin, cout;  // cin padded to 16 for the first layer
    float *W = nullptr, *b = nullptr, *gW = nullptr, *gb = nullptr, *mW = nullptr, *vW = nullptr, *mb = nullptr,
          *vb = nullptr;
    bf16 *Wb = nullptr, *Wt = nullptr;
  };
  Layer L[15];  // 14 convolutions + the 1x1 head (index 14)
  // activations (BF16, channels-last) and their gradients
  bf16 *x16 = nullptr, *e[3][2] = {}, *pl[3] = {}, *bt[2] = {}, *cat[3] = {}, *dc[3][2] = {};
  bf16 *gx16 = nullptr, *ge[3][2] = {}, *gpl[3] = {}, *gbt[2] = {}, *gcat[3] = {}, *gdc[3][2] = {};
  float* y = nullptr;
  double* part = nullptr;
  double* hpart = nullptr;
  long long step = 0;
  long long nlaunch_fwd = 0;  // kernel launches of one forward pass
  int tensor_path = 0;        // 0: mma.sync convolutions, 1: tcgen05 (TMEM accumulators)
  int* tc_err = nullptr;      // device flag: a tcgen05 wait gave up
  std::vector<void*> allocs;
  std::string err;
};

namespace {

using hb::kThreads;
using namespace hb::nn;

template <typename T>
int nalloc(hbf_unet* N, T** p, long long count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (size_t)(count > 0 ? count : 1) * sizeof(T)) != cudaSuccess) return HBF_ERR_OOM;
  N->allocs.push_back(q);
  if (cudaMemsetAsync(q, 0, (size_t)(count > 0 ? count : 1) * sizeof(T), N->stream) != cudaSuccess)
    return HBF_ERR_CUDA;
  *p = (T*)q;
  return HBF_OK;
}

int grid(long long n) { return hb::grid_for(n, 152 * 16); }

int taps(int d) { return d == 3 ? 27 : 9; }

void conv(hbf_unet* N, int lev, const bf16* in, int cin, const bf16* W, const float* b, int cout, bf16* out,
          int ostride, int ooff, int relu) {
  if (N->tensor_path == 1 && cin % 16 == 0 && cout % 16 == 0 && cout >= 16 && cout <= 256 && N->tc_err) {
    const Box bx = N->box[lev];
    const int hsmem = tc_halo_smem_bytes(N->d, cin, cout);
    if (bx.X % 8 == 0 && hsmem <= kTcHaloMaxSmem) {
      // every tap in shared memory: one MMA stream per CTA of 8 x 16 points
      const int blocks = (bx.X / 8) * ((bx.Y + 15) / 16) * bx.Z;
      if (N->d == 3)
        k_conv_fwd_tc_halo<3><<<blocks, kTcM, hsmem, N->stream>>>(in, cin, W, b, cout, out, ostride, ooff, relu,
                                                                  bx, tc_cols(cout), N->tc_err);
      else
        k_conv_fwd_tc_halo<2><<<blocks, kTcM, hsmem, N->stream>>>(in, cin, W, b, cout, out, ostride, ooff, relu,
                                                                  bx, tc_cols(cout), N->tc_err);
      return;
    }
    const int blocks = (int)((N->P[lev] + kTcM - 1) / kTcM);
    const int smem = tc_smem_bytes(cin, cout);
    if (N->d == 3)
      k_conv_fwd_tc<3><<<blocks, kTcM, smem, N->stream>>>(in, cin, W, b, cout, out, ostride, ooff, relu, bx,
                                                          tc_cols(cout), N->tc_err);
    else
      k_conv_fwd_tc<2><<<blocks, kTcM, smem, N->stream>>>(in, cin, W, b, cout, out, ostride, ooff, relu, bx,
                                                          tc_cols(cout), N->tc_err);
    return;
  }
  const int NT = cout / 8;
  const int NTB = NT <= 8 ? NT : (NT % 8 == 0 ? 8 : (NT % 6 == 0 ? 6 : 4));
  dim3 g((unsigned)((N->P[lev] + 63) / 64), (unsigned)(NT / NTB), 1);
  const Box bx = N->box[lev];
#define HB_CONV(DD, NN) k_conv_fwd<DD, NN><<<g, 128, 0, N->stream>>>(in, cin, W, b, cout, out, ostride, ooff, relu, bx)
  if (N->d == 3) {
    if (NTB == 2) HB_CONV(3, 2); else if (NTB == 4) HB_CONV(3, 4); else if (NTB == 6) HB_CONV(3, 6); else HB_CONV(3, 8);
  } else {
    if (NTB == 2) HB_CONV(2, 2); else if (NTB == 4) HB_CONV(2, 4); else if (NTB == 6) HB_CONV(2, 6); else HB_CONV(2, 8);
  }
#undef HB_CONV
}

void wgrad(hbf_unet* N, int lev, const bf16* x, int cin, const bf16* gz, int cout, float* gW) {
  const int chunk = 4096;
  const int pairs = (cin / 8) * (cout / 16);
  dim3 g((unsigned)((pairs + 3) / 4), (unsigned)taps(N->d), (unsigned)((N->P[lev] + chunk - 1) / chunk));
  if (N->d == 3)
    k_conv_wgrad<3><<<g, 128, 0, N->stream>>>(x, cin, gz, cout, gW, N->box[lev], chunk);
  else
    k_conv_wgrad<2><<<g, 128, 0, N->stream>>>(x, cin, gz, cout, gW, N->box[lev], chunk);
}

// backward of conv layer k (input `in` at level lev, output gradient g_out in
// place): ReLU mask, bias and weight gradients, input gradient into g_in
// (skipped when null)
void layer_back(hbf_unet* N, int k, int lev, const bf16* in, const bf16* out, bf16* g_out, bf16* g_in) {
  auto& Ly = N->L[k];
  const long long n = N->P[lev] * Ly.cout;
  k_relu_bwd<<<grid(n), kThreads, 0, N->stream>>>(g_out, out, n);
  k_bias_grad<<<grid(N->P[lev] / 8 + 1), 256, 256 * sizeof(float), N->stream>>>(g_out, Ly.cout, N->P[lev], Ly.gb);
  wgrad(N, lev, in, Ly.cin, g_out, Ly.cout, Ly.gW);
  if (g_in) conv(N, lev, g_out, Ly.cout, Ly.Wt, nullptr, Ly.cin, g_in, Ly.cin, 0, 0);
}

void refresh_bf16(hbf_unet* N) {
  for (int k = 0; k < 14; ++k) {
    auto& Ly = N->L[k];
    const long long n = (long long)taps(N->d) * Ly.cout * Ly.cin;
    k_f32_to_bf16<<<grid(n), kThreads, 0, N->stream>>>(Ly.Wb, Ly.W, n);
    if (N->d == 3)
      k_flip_transpose<3><<<grid(n), kThreads, 0, N->stream>>>(Ly.Wb, Ly.Wt, Ly.cout, Ly.cin);
    else
      k_flip_transpose<2><<<grid(n), kThreads, 0, N->stream>>>(Ly.Wb, Ly.Wt, Ly.cout, Ly.cin);
  }
}

void forward(hbf_unet* N, const float* x) {
  const int c0 = kCh[0], c1 = kCh[1], c2 = kCh[2], c3 = kCh[3];
  auto* L = N->L;
  k_pack_input<<<grid(N->P[0] * 16), kThreads, 0, N->stream>>>(N->x16, x, N->P[0]);
  const bf16* h = N->x16;
  for (int l = 0; l < 3; ++l) {
    conv(N, l, h, L[2 * l].cin, L[2 * l].Wb, L[2 * l].b, L[2 * l].cout, N->e[l][0], L[2 * l].cout, 0, 1);
    conv(N, l, N->e[l][0], L[2 * l + 1].cin, L[2 * l + 1].Wb, L[2 * l + 1].b, L[2 * l + 1].cout, N->e[l][1],
         L[2 * l + 1].cout, 0, 1);
    const int C = kCh[l];
    const long long n = N->P[l + 1] * C;
    if (N->d == 3)
      k_pool<3><<<grid(n), kThreads, 0, N->stream>>>(N->e[l][1], N->pl[l], C, N->box[l]);
    else
      k_pool<2><<<grid(n), kThreads, 0, N->stream>>>(N->e[l][1], N->pl[l], C, N->box[l]);
    h = N->pl[l];
  }
  conv(N, 3, N->pl[2], c2, L[6].Wb, L[6].b, c3, N->bt[0], c3, 0, 1);
  conv(N, 3, N->bt[0], c3, L[7].Wb, L[7].b, c3, N->bt[1], c3, 0, 1);
  const bf16* up = N->bt[1];
  int cup = c3;
  const int cs[3] = {c0, c1, c2};
  for (int l = 2; l >= 0; --l) {
    const int Cs = cup + cs[l];
    const long long n = N->P[l] * cup;
    if (N->d == 3)
      k_upsample<3><<<grid(n), kThreads, 0, N->stream>>>(up, cup, N->cat[l], Cs, N->box[l]);
    else
      k_upsample<2><<<grid(n), kThreads, 0, N->stream>>>(up, cup, N->cat[l], Cs, N->box[l]);
    k_copy_channels<<<grid(N->P[l] * cs[l]), kThreads, 0, N->stream>>>(N->e[l][1], cs[l], N->cat[l], Cs, cup,
                                                                        N->P[l]);
    const int ka = 8 + 2 * (2 - l), kb = ka + 1;
    conv(N, l, N->cat[l], Cs, L[ka].Wb, L[ka].b, cs[l], N->dc[l][0], cs[l], 0, 1);
    conv(N, l, N->dc[l][0], cs[l], L[kb].Wb, L[kb].b, cs[l], N->dc[l][1], cs[l], 0, 1);
    up = N->dc[l][1];
    cup = cs[l];
  }
  k_head_fwd<<<grid(N->P[0]), kThreads, 0, N->stream>>>(N->dc[0][1], L[14].W, L[14].b, N->y, N->P[0]);
}

void backward(hbf_unet* N, const float* gy) {
  const int c3 = kCh[3];
  auto* L = N->L;
  k_head_bwd<<<grid(N->P[0]), kThreads, 0, N->stream>>>(N->dc[0][1], L[14].W, gy, N->gdc[0][1], L[14].gW,
                                                         L[14].gb, N->P[0]);
  const int cs[3] = {kCh[0], kCh[1], kCh[2]};
  // decoder levels 0, 1, 2
  for (int l = 0; l < 3; ++l) {
    const int ka = 8 + 2 * (2 - l), kb = ka + 1;
    const int cup = l == 2 ? c3 : cs[l + 1];
    const int Cs = cup + cs[l];
    layer_back(N, kb, l, N->dc[l][0], N->dc[l][1], N->gdc[l][1], N->gdc[l][0]);
    layer_back(N, ka, l, N->cat[l], N->dc[l][0], N->gdc[l][0], N->gcat[l]);
    bf16* gup = l == 2 ? N->gbt[1] : N->gdc[l + 1][1];
    const long long n = N->P[l + 1] * cup;
    if (N->d == 3)
      k_upsample_bwd<3><<<grid(n), kThreads, 0, N->stream>>>(N->gcat[l], Cs, cup, gup, N->box[l]);
    else
      k_upsample_bwd<2><<<grid(n), kThreads, 0, N->stream>>>(N->gcat[l], Cs, cup, gup, N->box[l]);
  }
  // bottleneck
  layer_back(N, 7, 3, N->bt[0], N->bt[1], N->gbt[1], N->gbt[0]);
  layer_back(N, 6, 3, N->pl[2], N->bt[0], N->gbt[0], N->gpl[2]);
  // encoder levels 2, 1, 0
  for (int l = 2; l >= 0; --l) {
    const int cup = l == 2 ? c3 : cs[l + 1];
    const int Cs = cup + cs[l];
    const long long n = N->P[l] * cs[l];
    if (N->d == 3)
      k_pool_bwd_add<3><<<grid(n), kThreads, 0, N->stream>>>(N->gpl[l], N->gcat[l], Cs, cup, N->ge[l][1], cs[l],
                                                             N->box[l]);
    else
      k_pool_bwd_add<2><<<grid(n), kThreads, 0, N->stream>>>(N->gpl[l], N->gcat[l], Cs, cup, N->ge[l][1], cs[l],
                                                             N->box[l]);
    layer_back(N, 2 * l + 1, l, N->e[l][0], N->e[l][1], N->ge[l][1], N->ge[l][0]);
    const bf16* in = l == 0 ? N->x16 : N->pl[l - 1];
    bf16* gin = l == 0 ? nullptr : N->gpl[l - 1];
    layer_back(N, 2 * l, l, in, N->e[l][0], N->ge[l][0], gin);
  }
}

int check(hbf_unet* N, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return HBF_OK;
  N->err = std::string(what) + ": " + cudaGetErrorString(e);
  return HBF_ERR_CUDA;
}

}  // namespace

// ---------------------------------------------------------------------------
// the guess inside the nodal projection
// ---------------------------------------------------------------------------
namespace {

// x[point] = r[node] * scale on the nodes, 0 in the padding
__global__ void k_nodes_to_net(const double* __restrict__ r, double scale, int e0, int e1, int e2, Box box,
                               float* __restrict__ x) {
  const long long P = (long long)box.X * box.Y * box.Z;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    coords(box, t, i, j, k);
    x[t] = (i < e0 && j < e1 && k < e2) ? (float)(r[i + (long long)e0 * (j + (long long)e1 * k)] * scale) : 0.f;
  }
}

// delta[node] = y[point]
__global__ void k_net_to_nodes(const float* __restrict__ y, int e0, int e1, int e2, Box box, double* __restrict__ out) {
  const long long n = (long long)e0 * e1 * e2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % e0);
    const long long r = t / e0;
    const int j = (int)(r % e1), k = (int)(r / e1);
    out[t] = (double)y[i + (long long)box.X * (j + (long long)box.Y * k)];
  }
}

}  // namespace

namespace hb {

// 1 if a tcgen05 convolution of N gave up waiting for the tensor cores
// since the flag was last cleared (then clears it); synchronises stream s
int take_tc_err(hbf_unet* N, cudaStream_t s) {
  if (!N->tc_err) return 0;
  int h = 0;
  if (cudaMemcpyAsync(&h, N->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 1;
  if (h) cudaMemsetAsync(N->tc_err, 0, sizeof(int), s);
  return h != 0;
}

// x[point] = r[cell] * scale (FP32 cells), 0 in the padding
__global__ void k_cells_to_net_f(const float* __restrict__ r, float scale, int e0, int e1, int e2, Box box,
                                 float* __restrict__ x) {
  const long long P = (long long)box.X * box.Y * box.Z;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < P; t += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    coords(box, t, i, j, k);
    x[t] = (i < e0 && j < e1 && k < e2) ? r[i + (long long)e0 * (j + (long long)e1 * k)] * scale : 0.f;
  }
}

__global__ void k_net_to_cells_f(const float* __restrict__ y, int e0, int e1, int e2, Box box, float* __restrict__ out) {
  const long long n = (long long)e0 * e1 * e2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % e0);
    const long long r = t / e0;
    const int j = (int)(r % e1), k = (int)(r / e1);
    out[t] = y[i + (long long)box.X * (j + (long long)box.Y * k)];
  }
}

// The network's direction for the viscous residual: each velocity component
// of r32 (scaled by `scale`) restricted to the network's level by cell
// averaging, one forward pass per component, the outputs interpolated back
// to the finest cells (multilinear, odd reflection at the walls).  The level
// arrays of the FP32 V-cycles serve as scratch (the solve has not started).
bool visc_net_direction(hbf_ctx* c, const float* r32, double scale, float* d32) {
  hbf_unet* N = c->vnet;
  if (!N || !c->vnet_x) return false;
  const int L = c->vnet_level;
  const float* src = r32;
  for (int l = 0; l < L; ++l) {
    cell_restrict_f(c, l, src, c->lv[l + 1].fvb);
    src = c->lv[l + 1].fvb;
  }
  const Geom& gL = c->lv[L].g;
  const int e0 = gL.n[0], e1 = gL.n[1], e2 = c->dim == 3 ? gL.n[2] : 1;
  float* outL = L == 0 ? d32 : c->lv[L].fvx;
  cudaStream_t saved = N->stream;
  N->stream = c->stream;
  for (int q = 0; q < c->dim; ++q) {
    k_cells_to_net_f<<<grid(N->P[0]), kThreads, 0, c->stream>>>(src + (size_t)q * gL.ncell, (float)scale, e0, e1, e2,
                                                                 N->box[0], c->vnet_x);
    forward(N, c->vnet_x);
    k_net_to_cells_f<<<grid((long long)gL.ncell), kThreads, 0, c->stream>>>(N->y, e0, e1, e2, N->box[0],
                                                                           outL + (size_t)q * gL.ncell);
    c->nlaunch += N->nlaunch_fwd + 2;
  }
  N->stream = saved;
  for (int l = L - 1; l >= 0; --l) {
    float* fine = l == 0 ? d32 : c->lv[l].fvx;
    cudaMemsetAsync(fine, 0, sizeof(float) * (size_t)c->dim * c->lv[l].g.ncell, c->stream);
    cell_prolong_add_f(c, l, fine, c->lv[l + 1].fvx);
  }
  if (cudaGetLastError() != cudaSuccess) return false;
  // a convolution that gave up waiting on the tensor cores left its output
  // partly unwritten: no direction this step
  return !take_tc_err(N, c->stream);
}

void release_visc_guess(hbf_ctx* c) {
  if (c->vnet_x) cudaFree(c->vnet_x);
  c->vnet_x = nullptr;
  c->vnet = nullptr;
}

void release_guess(hbf_ctx* c) {
  if (c->ntry) cudaFree(c->ntry);
  if (c->nzero) cudaFree(c->nzero);
  if (c->net_x) cudaFree(c->net_x);
  c->ntry = nullptr;
  c->nzero = nullptr;
  c->net_x = nullptr;
  c->guess = nullptr;
}

// Candidate p + alpha delta, delta = the network's correction for the
// normalised warm-start residual r0, alpha the least-squares step
// argmin |r0 - alpha L delta|_2; kept only if its max-norm residual is smaller.
int apply_guess(hbf_ctx* c, const double* b, double* p, int* used) {
  (void)b;
  const ProfRegion region(c, kSlotGuess);
  *used = 0;
  hbf_unet* N = c->guess;
  int st = 0;
  const long long nn = c->g.nnode;
  const double n0 = reduce_max_abs(c, c->nres0, nn, &st);
  if (st) return st;
  if (!(n0 > 0.0) || !std::isfinite(n0)) return HBF_OK;
  // the network sees the warm-start residual on the nodes of level L
  // (full weighting down from the finest level) and its output is
  // interpolated back up, level by level
  const int L = c->guess_level;
  const double* src = c->nres0;
  for (int l = 0; l < L; ++l) {
    nodal_restrict(c, l, src, c->lv[l + 1].nb);
    src = c->lv[l + 1].nb;
  }
  const Geom& gL = c->lv[L].g;
  const int e0 = gL.n[0] + 1, e1 = gL.n[1] + 1, e2 = c->dim == 3 ? gL.n[2] + 1 : 1;
  cudaStream_t saved = N->stream;
  N->stream = c->stream;
  k_nodes_to_net<<<grid(N->P[0]), kThreads, 0, c->stream>>>(src, 1.0 / n0, e0, e1, e2, N->box[0], c->net_x);
  forward(N, c->net_x);
  N->stream = saved;
  double* outL = L == 0 ? c->ntry : c->lv[L].nx;
  k_net_to_nodes<<<grid((long long)gL.nnode), kThreads, 0, c->stream>>>(N->y, e0, e1, e2, N->box[0], outL);
  c->nlaunch += N->nlaunch_fwd + 2;
  for (int l = L - 1; l >= 0; --l) {
    double* fine = l == 0 ? c->ntry : c->lv[l].nx;
    if ((st = cuda_check(c, cudaMemsetAsync(fine, 0, (size_t)c->lv[l].g.nnode * sizeof(double), c->stream),
                         "learned guess")))
      return st;
    nodal_prolong_add(c, l, fine, c->lv[l + 1].nx);
  }
  if ((st = cuda_check(c, cudaGetLastError(), "learned guess"))) return st;
  // w = -L delta, alpha = -(r0, w)/(w, w), candidate residual r0 + alpha w
  double* w = c->lv[0].nr;
  double* rtry = c->lv[0].nb;
  if ((st = nodal_residual(c, c->nzero, c->ntry, w))) return st;
  const double rw = reduce_dot(c, c->nres0, w, nn, &st);
  if (st) return st;
  const double ww = reduce_dot(c, w, w, nn, &st);
  if (st) return st;
  if (!(ww > 0.0) || !std::isfinite(rw)) return HBF_OK;
  // a tcgen05 convolution that gave up waiting left part of the output
  // unwritten: discard the candidate (the solve starts from p) and clear
  // the flag (the reductions above have synchronised the stream)
  if (take_tc_err(N, c->stream)) return HBF_OK;
  const double alpha = -rw / ww;
  axmy(c, rtry, c->nres0, -alpha, w, nn);
  const double n1 = reduce_max_abs(c, rtry, nn, &st);
  if (st) return st;
  if (n1 < n0) {
    axmy(c, p, p, -alpha, c->ntry, nn);
    *used = 1;
  }
  return cuda_check(c, cudaGetLastError(), "learned guess");
}

}  // namespace hb

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

int hbf_unet_create(hbf_unet** out, int dim, const int64_t n[3], int train, uint64_t seed, void* stream) {
  if (!out || !n || (dim != 2 && dim != 3)) return HBF_ERR_ARG;
  *out = nullptr;
  for (int a = 0; a < dim; ++a)
    if (n[a] < 8 || n[a] % 8 != 0 || n[a] > 4096) return HBF_ERR_ARG;
  hbf_unet* N = new (std::nothrow) hbf_unet();
  if (!N) return HBF_ERR_OOM;
  N->d = dim;
  N->train = train != 0;
  N->nlaunch_fwd = 25;  // pack, 14 convolutions, 3 pools, 3 upsamples, 3 copies, head
  N->stream = (cudaStream_t)stream;
  for (int l = 0; l < 4; ++l) {
    const int s = 1 << l;
    N->box[l] = Box{(int)(n[0] / s), (int)(n[1] / s), dim == 3 ? (int)(n[2] / s) : 1};
    N->P[l] = (long long)N->box[l].X * N->box[l].Y * N->box[l].Z;
  }
  const int c0 = kCh[0], c1 = kCh[1], c2 = kCh[2], c3 = kCh[3];
  const int shapes[14][2] = {{16, c0}, {c0, c0}, {c0, c1}, {c1, c1}, {c1, c2}, {c2, c2}, {c2, c3},
                             {c3, c3}, {c3 + c2, c2}, {c2, c2}, {c2 + c1, c1}, {c1, c1}, {c1 + c0, c0}, {c0, c0}};
  const int T = taps(dim);
  int st = HBF_OK;
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
#define NA(p, c) \
  if ((st = nalloc(N, &(p), (c)))) goto fail
  for (int k = 0; k < 15; ++k) {
    auto& Ly = N->L[k];
    Ly.cin = k < 14 ? shapes[k][0] : 16;
    Ly.cout = k < 14 ? shapes[k][1] : 1;
    const long long nw = k < 14 ? (long long)T * Ly.cout * Ly.cin : 16;
    NA(Ly.W, nw);
    NA(Ly.b, Ly.cout);
    if (k < 14) {
      NA(Ly.Wb, nw);
      NA(Ly.Wt, nw);
    }
    if (N->train) {
      NA(Ly.gW, nw);
      NA(Ly.gb, Ly.cout);
      NA(Ly.mW, nw);
      NA(Ly.vW, nw);
      NA(Ly.mb, Ly.cout);
      NA(Ly.vb, Ly.cout);
    }
    // He-normal initial weights (the first layer's padded input channels stay 0)
    std::vector<float> h((size_t)nw, 0.f);
    const int fan_in = k < 14 ? T * (k == 0 ? 1 : Ly.cin) : 16;
    const double sd = std::sqrt((k < 14 ? 2.0 : 1.0) / fan_in);
    for (long long q = 0; q < nw; ++q) {
      const int ci = (int)(q % Ly.cin);
      h[(size_t)q] = (k == 0 && ci != 0) ? 0.f : (float)(nd(rng) * sd);
    }
    if (cudaMemcpyAsync(Ly.W, h.data(), (size_t)nw * sizeof(float), cudaMemcpyHostToDevice, N->stream) !=
        cudaSuccess) {
      st = HBF_ERR_CUDA;
      goto fail;
    }
  }
  NA(N->tc_err, 1);
  NA(N->x16, N->P[0] * 16);
  for (int l = 0; l < 3; ++l) {
    NA(N->e[l][0], N->P[l] * kCh[l]);
    NA(N->e[l][1], N->P[l] * kCh[l]);
    NA(N->pl[l], N->P[l + 1] * kCh[l]);
    const int cup = l == 2 ? c3 : kCh[l + 1];
    NA(N->cat[l], N->P[l] * (cup + kCh[l]));
    NA(N->dc[l][0], N->P[l] * kCh[l]);
    NA(N->dc[l][1], N->P[l] * kCh[l]);
    if (N->train) {
      NA(N->ge[l][0], N->P[l] * kCh[l]);
      NA(N->ge[l][1], N->P[l] * kCh[l]);
      NA(N->gpl[l], N->P[l + 1] * kCh[l]);
      NA(N->gcat[l], N->P[l] * (cup + kCh[l]));
      NA(N->gdc[l][0], N->P[l] * kCh[l]);
      NA(N->gdc[l][1], N->P[l] * kCh[l]);
    }
  }
  NA(N->bt[0], N->P[3] * c3);
  NA(N->bt[1], N->P[3] * c3);
  if (N->train) {
    NA(N->gbt[0], N->P[3] * c3);
    NA(N->gbt[1], N->P[3] * c3);
  }
  NA(N->y, N->P[0]);
  NA(N->part, 2432);
#undef NA
  if (cudaMallocHost((void**)&N->hpart, 2432 * sizeof(double)) != cudaSuccess) {
    st = HBF_ERR_OOM;
    goto fail;
  }
  refresh_bf16(N);
  if ((st = check(N, "unet init"))) goto fail;
  if (cudaStreamSynchronize(N->stream) != cudaSuccess) {
    st = HBF_ERR_CUDA;
    goto fail;
  }
  // tcgen05 convolutions by default (mma.sync if their launch attribute fails)
  if (hbf_unet_set_tensor_path(N, 1) != HBF_OK) N->tensor_path = 0;
  *out = N;
  return HBF_OK;
fail:
  hbf_unet_destroy(N);
  return st;
}

void hbf_unet_destroy(hbf_unet* N) {
  if (!N) return;
  cudaStreamSynchronize(N->stream);
  for (void* p : N->allocs) cudaFree(p);
  if (N->hpart) cudaFreeHost(N->hpart);
  delete N;
}

const char* hbf_unet_last_error(const hbf_unet* N) { return N ? N->err.c_str() : "null network"; }

int64_t hbf_unet_param_count(const hbf_unet* N) {
  if (!N) return HBF_ERR_ARG;
  int64_t s = 0;
  for (int k = 0; k < 15; ++k) s += (k < 14 ? (int64_t)taps(N->d) * N->L[k].cout * N->L[k].cin : 16) + N->L[k].cout;
  return s;
}

static int copy_params(hbf_unet* N, float* host_or_dev, int which, bool in) {
  if (!N || !host_or_dev) return HBF_ERR_ARG;
  if ((which == 1) && !N->train) return HBF_ERR_ARG;
  long long off = 0;
  for (int k = 0; k < 15; ++k) {
    auto& Ly = N->L[k];
    const long long nw = k < 14 ? (long long)taps(N->d) * Ly.cout * Ly.cin : 16;
    float* w = which == 0 ? Ly.W : Ly.gW;
    float* b = which == 0 ? Ly.b : Ly.gb;
    const cudaMemcpyKind kd = cudaMemcpyDefault;
    cudaError_t e1 = in ? cudaMemcpyAsync(w, host_or_dev + off, nw * sizeof(float), kd, N->stream)
                        : cudaMemcpyAsync(host_or_dev + off, w, nw * sizeof(float), kd, N->stream);
    off += nw;
    cudaError_t e2 = in ? cudaMemcpyAsync(b, host_or_dev + off, Ly.cout * sizeof(float), kd, N->stream)
                        : cudaMemcpyAsync(host_or_dev + off, b, Ly.cout * sizeof(float), kd, N->stream);
    off += Ly.cout;
    if (e1 != cudaSuccess || e2 != cudaSuccess) return HBF_ERR_CUDA;
  }
  if (in && which == 0) refresh_bf16(N);
  if (cudaStreamSynchronize(N->stream) != cudaSuccess) return HBF_ERR_CUDA;
  return check(N, "unet params");
}

int hbf_unet_get_params(hbf_unet* N, float* dst) { return copy_params(N, dst, 0, false); }
int hbf_unet_set_params(hbf_unet* N, const float* src) { return copy_params(N, const_cast<float*>(src), 0, true); }
int hbf_unet_get_grads(hbf_unet* N, float* dst) { return copy_params(N, dst, 1, false); }

int hbf_unet_set_tensor_path(hbf_unet* N, int path) {
  if (!N || (path != 0 && path != 1)) return HBF_ERR_ARG;
  if (path == 1) {
    // the largest tile: 128 points plus 256 output channels, of 256 input channels
    const int bytes = tc_smem_bytes(256, 256);
    if (cudaFuncSetAttribute(k_conv_fwd_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_fwd_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_fwd_tc_halo<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcHaloMaxSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_conv_fwd_tc_halo<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcHaloMaxSmem) !=
            cudaSuccess) {
      cudaGetLastError();
      N->err = "tcgen05 convolution: shared-memory attribute";
      return HBF_ERR_CUDA;
    }
  }
  N->tensor_path = path;
  return HBF_OK;
}


int hbf_unet_tensor_status(hbf_unet* N) {
  if (!N) return HBF_ERR_ARG;
  int h = 0;
  if (cudaMemcpyAsync(&h, N->tc_err, sizeof(int), cudaMemcpyDeviceToHost, N->stream) != cudaSuccess ||
      cudaStreamSynchronize(N->stream) != cudaSuccess)
    return HBF_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(N->tc_err, 0, sizeof(int), N->stream);
    N->err = "a tcgen05 convolution gave up waiting for the tensor cores";
    return HBF_ERR_TIMEOUT;
  }
  return HBF_OK;
}

int hbf_unet_forward(hbf_unet* N, const float* x_dev, float* y_dev) {
  if (!N || !x_dev) return HBF_ERR_ARG;
  forward(N, x_dev);
  if (y_dev && cudaMemcpyAsync(y_dev, N->y, N->P[0] * sizeof(float), cudaMemcpyDeviceToDevice, N->stream) !=
                   cudaSuccess)
    return HBF_ERR_CUDA;
  return check(N, "unet forward");
}

int hbf_unet_backward(hbf_unet* N, const float* gy_dev) {
  if (!N || !gy_dev || !N->train) return HBF_ERR_ARG;
  backward(N, gy_dev);
  return check(N, "unet backward");
}

int hbf_unet_loss(hbf_unet* N, const float* t_dev, const float* mask_dev, float* gy_dev, double* loss) {
  if (!N || !t_dev || !mask_dev || !gy_dev || !loss) return HBF_ERR_ARG;
  const int nb = 2432;
  // number of valid points: the mask's sum
  k_mask_sum<<<nb, kThreads, 0, N->stream>>>(mask_dev, N->part, N->P[0]);
  if (cudaMemcpyAsync(N->hpart, N->part, nb * sizeof(double), cudaMemcpyDeviceToHost, N->stream) != cudaSuccess ||
      cudaStreamSynchronize(N->stream) != cudaSuccess)
    return HBF_ERR_CUDA;
  double nvalid = 0.0;
  for (int q = 0; q < nb; ++q) nvalid += N->hpart[q];
  if (!(nvalid > 0.0)) return HBF_ERR_ARG;
  k_mse<<<nb, kThreads, 0, N->stream>>>(N->y, t_dev, mask_dev, gy_dev, N->part, N->P[0], 1.0 / nvalid);
  if (cudaMemcpyAsync(N->hpart, N->part, nb * sizeof(double), cudaMemcpyDeviceToHost, N->stream) != cudaSuccess ||
      cudaStreamSynchronize(N->stream) != cudaSuccess)
    return HBF_ERR_CUDA;
  double s = 0.0;
  for (int q = 0; q < nb; ++q) s += N->hpart[q];
  *loss = s;
  // the loss is the first synchronising call after a training forward pass:
  // a tensor-core wait that gave up there invalidates this output
  if (hb::take_tc_err(N, N->stream)) {
    N->err = "a tcgen05 convolution gave up waiting for the tensor cores";
    return HBF_ERR_TIMEOUT;
  }
  return check(N, "unet loss");
}

int hbf_unet_adam(hbf_unet* N, double lr, double b1, double b2, double eps) {
  if (!N || !N->train || !(lr > 0.0)) return HBF_ERR_ARG;
  ++N->step;
  const float c1 = (float)(1.0 - std::pow(b1, (double)N->step)), c2 = (float)(1.0 - std::pow(b2, (double)N->step));
  for (int k = 0; k < 15; ++k) {
    auto& Ly = N->L[k];
    const long long nw = k < 14 ? (long long)taps(N->d) * Ly.cout * Ly.cin : 16;
    k_adam<<<grid(nw), kThreads, 0, N->stream>>>(Ly.W, Ly.gW, Ly.mW, Ly.vW, k < 14 ? Ly.Wb : nullptr, nw, (float)lr,
                                                  (float)b1, (float)b2, (float)eps, c1, c2);
    k_adam<<<grid(Ly.cout), kThreads, 0, N->stream>>>(Ly.b, Ly.gb, Ly.mb, Ly.vb, nullptr, Ly.cout, (float)lr,
                                                       (float)b1, (float)b2, (float)eps, c1, c2);
  }
  // (the first layer's padded input channels have zero gradient and stay zero)
  refresh_bf16(N);
  return check(N, "unet adam");
}

int hbf_set_visc_guess_model(hbf_ctx* c, hbf_unet* N, int level) {
  if (!c) return HBF_ERR_ARG;
  hb::release_visc_guess(c);
  if (!N) return HBF_OK;
  if (c->precision != HBF_MIXED) return hb::fail(c, HBF_ERR_ARG, "the viscous guess needs a mixed context");
  if (N->d != c->dim) return hb::fail(c, HBF_ERR_ARG, "guess model dimension differs from the grid's");
  if (level < 0 || level >= (int)c->lv.size())
    return hb::fail(c, HBF_ERR_ARG, "guess level outside the multigrid hierarchy");
  const hb::Geom& gL = c->lv[level].g;
  const int e[3] = {gL.n[0], gL.n[1], c->dim == 3 ? gL.n[2] : 1};
  const int b[3] = {N->box[0].X, N->box[0].Y, N->box[0].Z};
  for (int a = 0; a < c->dim; ++a)
    if (b[a] < e[a]) return hb::fail(c, HBF_ERR_ARG, "guess model box is smaller than the cell grid");
  if (cudaMalloc((void**)&c->vnet_x, (size_t)N->P[0] * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    c->vnet_x = nullptr;
    return hb::fail(c, HBF_ERR_OOM, "guess buffers");
  }
  c->vnet = N;
  c->vnet_level = level;
  return HBF_OK;
}

int hbf_set_guess_model(hbf_ctx* c, hbf_unet* N) { return hbf_set_guess_model_level(c, N, 0); }

int hbf_set_guess_model_level(hbf_ctx* c, hbf_unet* N, int level) {
  if (!c) return HBF_ERR_ARG;
  hb::release_guess(c);
  if (!N) return HBF_OK;
  if (N->d != c->dim) return hb::fail(c, HBF_ERR_ARG, "guess model dimension differs from the grid's");
  if (level < 0 || level >= (int)c->lv.size())
    return hb::fail(c, HBF_ERR_ARG, "guess level outside the multigrid hierarchy");
  const hb::Geom& gL = c->lv[level].g;
  const int e[3] = {gL.n[0] + 1, gL.n[1] + 1, c->dim == 3 ? gL.n[2] + 1 : 1};
  const int b[3] = {N->box[0].X, N->box[0].Y, N->box[0].Z};
  for (int a = 0; a < c->dim; ++a)
    if (b[a] < e[a]) return hb::fail(c, HBF_ERR_ARG, "guess model box is smaller than the node grid");
  if (cudaMalloc((void**)&c->ntry, (size_t)c->g.nnode * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->nzero, (size_t)c->g.nnode * sizeof(double)) != cudaSuccess ||
      cudaMemset(c->nzero, 0, (size_t)c->g.nnode * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->net_x, (size_t)N->P[0] * sizeof(float)) != cudaSuccess) {
    hb::release_guess(c);
    return hb::fail(c, HBF_ERR_OOM, "guess buffers");
  }
  c->guess = N;
  c->guess_level = level;
  return HBF_OK;
}

int hbf_unet_zero_grads(hbf_unet* N) {
  if (!N || !N->train) return HBF_ERR_ARG;
  for (int k = 0; k < 15; ++k) {
    auto& Ly = N->L[k];
    const long long nw = k < 14 ? (long long)taps(N->d) * Ly.cout * Ly.cin : 16;
    if (cudaMemsetAsync(Ly.gW, 0, nw * sizeof(float), N->stream) != cudaSuccess ||
        cudaMemsetAsync(Ly.gb, 0, Ly.cout * sizeof(float), N->stream) != cudaSuccess)
      return HBF_ERR_CUDA;
  }
  return HBF_OK;
}

}  // extern "C"
