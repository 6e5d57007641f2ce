// Multigrid solvers and reductions (host drivers + kernel instantiations).
//
// V(nu1, nu2) cycle, as stated for the three solves of Sec. III A:
//   nu1 smoothing sweeps; r = b - A x; restrict r to the next level's b;
//   x_coarse = 0; recurse; x += P x_coarse; nu2 sweeps.
//   coarsest level: nu_bottom sweeps in a single thread block.
//   stop when ||b - A x||_inf <= rtol ||b||_inf.
// Singular problems (MAC and nodal potentials) remove the (weighted) mean of
// the right-hand side and pin the mean of the iterate after each cycle and the
// bottom solve.
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <type_traits>

#include "hb_internal.h"
#include "hb_mg_kernels.cuh"
#include "hb_vcycle_tail.cuh"
#include "hb_visc_fused.cuh"
#include "hb_visc_split.cuh"
#include "hb_visc_tma.cuh"

#include <cudaTypedefs.h>

namespace hb {

// ---------------------------------------------------------------------------
// deterministic reductions: fixed grid, per-block partials, one final block
// ---------------------------------------------------------------------------
template <int MODE>  // 0: max |x| (non-finite -> +inf), 1: sum x, 2: weighted nodal sum
__global__ void k_reduce_partial(const double* __restrict__ x, long long n, double* __restrict__ part,
                                 const __grid_constant__ Geom g, int dim) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    double v = x[t];
    if (MODE == 0) {
      double a = fabs(v);
      if (!isfinite(a)) a = INFINITY;
      acc = fmax(acc, a);
    } else if (MODE == 1) {
      acc += v;
    } else {
      int e0 = g.n[0] + 1, e1 = g.n[1] + 1;
      int i = (int)(t % e0);
      int q = (int)(t / e0);
      int j = q % e1;
      int k = q / e1;
      double w = 1.0;
      w = node_weight(g, i, j, k, dim);
      acc += w * v;
    }
  }
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = MODE == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = MODE == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

template <int MODE>
__global__ void k_reduce_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc = MODE == 0 ? fmax(acc, part[t]) : acc + part[t];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = MODE == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = MODE == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) *out = v;
  }
}

// x -= (*sum) * inv_count  (mean removal without a host round trip)
template <typename T>
__global__ void k_sub_mean(T* __restrict__ x, long long n, const double* __restrict__ sum, double inv_count) {
  T m = T(*sum * inv_count);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] -= m;
}

// Elementwise kernels touch four elements per step with 16-byte accesses
// (one float4, or two double2) when every array is 16-byte aligned, which
// keeps several loads in flight per thread on the capped grids; the elements
// past the last whole group go to thread 0.  The arithmetic per element is
// the one-element form's.
template <typename T>
struct V4 {
  T v[4];
};
__device__ __forceinline__ V4<float> ld4(const float* p, long long q) {
  const float4 f = reinterpret_cast<const float4*>(p)[q];
  return {{f.x, f.y, f.z, f.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p, long long q) {
  const double2 a = reinterpret_cast<const double2*>(p)[2 * q], b = reinterpret_cast<const double2*>(p)[2 * q + 1];
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, long long q, const V4<float>& v) {
  reinterpret_cast<float4*>(p)[q] = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
__device__ __forceinline__ void st4(double* p, long long q, const V4<double>& v) {
  reinterpret_cast<double2*>(p)[2 * q] = make_double2(v.v[0], v.v[1]);
  reinterpret_cast<double2*>(p)[2 * q + 1] = make_double2(v.v[2], v.v[3]);
}
template <typename... P>
__device__ __forceinline__ bool aligned16_all(const P*... p) {
  return ((reinterpret_cast<uintptr_t>(p) | ...) & 15) == 0;
}
// grid-stride loop: f4(q) on the groups 4q .. 4q + 3 when vec, f1(e) on single
// elements otherwise (and on the tail)
template <typename F4, typename F1>
__device__ __forceinline__ void for_each4(long long n, bool vec, F4 f4, F1 f1) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (vec) {
    const long long n4 = n >> 2;
#pragma unroll 4
    for (long long q = tid; q < n4; q += T) f4(q);
    if (tid == 0)
      for (long long e = n4 << 2; e < n; ++e) f1(e);
  } else {
    for (long long e = tid; e < n; e += T) f1(e);
  }
}

template <typename T>
__global__ void k_zero(T* __restrict__ x, long long n) {
  for_each4(
      n, aligned16_all(x), [&](long long q) { st4(x, q, V4<T>{{T(0), T(0), T(0), T(0)}}); },
      [&](long long e) { x[e] = T(0); });
}

__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, long long n,
                              double* __restrict__ part) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    acc += a[t] * b[t];
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// Vectorised partials of the frequent reductions: 16-byte loads, four
// iterations unrolled so that each thread keeps several loads in flight.
// Thread t takes the vectors t, t + T, t + 2T, ... (T threads in the grid) in
// that order, the tail past the last whole vector goes to thread 0, and the
// block and final sums run in a fixed order: the result is the same on every
// run.  MODE 0: max |x| (non-finite -> +inf); 1: sum x.  x 16-byte aligned.
template <int MODE>
__device__ __forceinline__ double red_op(double acc, double v) {
  if (MODE == 0) {
    double a = fabs(v);
    if (!isfinite(a)) a = INFINITY;
    return fmax(acc, a);
  }
  return acc + v;
}

template <int MODE>
__device__ __forceinline__ void block_partial(double acc, double* part) {
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = MODE == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = MODE == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

template <int MODE>
__global__ void k_reduce_partial_v(const double* __restrict__ x, long long n, double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n2 = n >> 1;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  double acc = 0.0;
#pragma unroll 4
  for (long long q = tid; q < n2; q += T) {
    const double2 v = x2[q];
    acc = red_op<MODE>(red_op<MODE>(acc, v.x), v.y);
  }
  if (tid == 0 && (n & 1)) acc = red_op<MODE>(acc, x[n - 1]);
  block_partial<MODE>(acc, part);
}

__global__ void k_dot_partial_v(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n2 = n >> 1;
  const double2* a2 = reinterpret_cast<const double2*>(a);
  const double2* b2 = reinterpret_cast<const double2*>(b);
  double acc = 0.0;
#pragma unroll 4
  for (long long q = tid; q < n2; q += T) {
    const double2 u = a2[q], v = b2[q];
    acc += u.x * v.x + u.y * v.y;
  }
  if (tid == 0 && (n & 1)) acc += a[n - 1] * b[n - 1];
  block_partial<1>(acc, part);
}

static inline bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }
static inline bool aligned8(const void* p) { return ((uintptr_t)p & 7) == 0; }

// a periodic axis: the Poisson and transfer kernels take their PER = true
// form (with the wraps); walls on every axis take PER = false
static inline bool any_per(const Geom& g) { return g.per[0] || g.per[1] || g.per[2]; }

// The FP32 finest level of the mixed viscous solve in the colour-split layout
// (hb_visc_split.cuh): 3D, walls on every axis, even n0, at least two levels,
// and none of the opt-in sweep or operator forms that read the natural layout
// (staged, fused) nor a network on level 0.  Every FP32 level-0 vector of the
// solve (the BiCGStab vectors, the V-cycle's level-0 arrays, the cell
// viscosity, the previous increment) is then split; FP64 arrays stay natural.
static bool split0(const hbf_ctx* c) {
  const Geom& g = c->g;
  return c->split_layout && c->dim == 3 && c->precision == HBF_MIXED && !any_per(g) && g.n[0] % 2 == 0 &&
         g.n[0] >= 4 && g.n[1] >= 3 && g.n[2] >= 3 && c->lv.size() >= 2 && c->lv[0].feta != nullptr &&
         !c->staged_tx && !c->staged_op_rows && !c->fused_sweep && !(c->vnet && c->vnet_level == 0);
}

template <int MODE>
static int reduce_to_device(hbf_ctx* c, const double* x, long long n, double* out) {
  if (MODE < 2 && aligned16(x))
    launch(c, kSlotReduce, k_reduce_partial_v<MODE < 2 ? MODE : 0>, kRedBlocks, kThreads, x, n, c->partial);
  else
    launch(c, kSlotReduce, k_reduce_partial<MODE>, kRedBlocks, kThreads, x, n, c->partial, c->g, c->dim);
  launch(c, kSlotReduce, k_reduce_final<MODE>, 1, 1024, c->partial, kRedBlocks, out);
  return cuda_check(c, cudaGetLastError(), "reduction");
}

static double read_result(hbf_ctx* c, const double* dev, int* st) {
  cudaError_t e = cudaMemcpyAsync(c->hres, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    *st = cuda_check(c, e, "reading a reduction");
    return NAN;
  }
  return *c->hres;
}

double reduce_max_abs(hbf_ctx* c, const double* x, long long n, int* st) {
  *st = reduce_to_device<0>(c, x, n, c->dres);
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

double reduce_dot(hbf_ctx* c, const double* a, const double* b, long long n, int* st) {
  if (aligned16(a) && aligned16(b))
    launch(c, kSlotReduce, k_dot_partial_v, kRedBlocks, kThreads, a, b, n, c->partial);
  else
    launch(c, kSlotReduce, k_dot_partial, kRedBlocks, kThreads, a, b, n, c->partial);
  launch(c, kSlotReduce, k_reduce_final<1>, 1, 1024, (const double*)c->partial, kRedBlocks, c->dres);
  *st = cuda_check(c, cudaGetLastError(), "dot");
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

double reduce_sum(hbf_ctx* c, const double* x, long long n, int* st) {
  *st = reduce_to_device<1>(c, x, n, c->dres);
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

// ---------------------------------------------------------------------------
// CFL time step without any device allocation (hbf_cfl_dt_noalloc)
// ---------------------------------------------------------------------------
// Callers that cannot allocate device memory -- code running inside a CUDA
// graph capture (where cudaMalloc is not allowed), hosts whose device memory is
// owned by another runtime's pool allocator, or embedded drivers that reserve
// all memory up front -- still need the time-step rule.  This variant of the
// max-|u| reduction keeps its per-block partials in a file-scope device array
// instead of the context's allocated scratch.  Every GPU that loads the
// library holds this array (256 KiB) until the process exits.
constexpr int kNoAllocBlocks = 32768;                       // partial slots
constexpr long long kNoAllocPerBlock = (long long)kThreads * 8;  // elements per block
constexpr long long kNoAllocMaxN = (long long)kNoAllocBlocks * kNoAllocPerBlock;
static __device__ __align__(256) double g_noalloc_partial[kNoAllocBlocks];

// one block per kNoAllocPerBlock elements: max |x| of its chunk (non-finite -> +inf)
__global__ void k_noalloc_maxabs_partial(const double* __restrict__ x, long long n, double* __restrict__ part) {
  long long base = (long long)blockIdx.x * kNoAllocPerBlock;
  double acc = 0.0;
  for (int q = 0; q < 8; ++q) {
    long long t = base + (long long)q * kThreads + threadIdx.x;
    if (t < n) {
      double a = fabs(x[t]);
      if (!isfinite(a)) a = INFINITY;
      acc = fmax(acc, a);
    }
  }
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// reduce the nb partials written by this call and write dt
__global__ void k_noalloc_cfl_final(const double* __restrict__ part, int nb, double h, double cfl,
                                    double* __restrict__ dt_out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc = fmax(acc, part[t]);
  for (int off = 16; off > 0; off >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    // every finite |u| is below +inf, so +inf marks a non-finite input: dt
    // becomes NaN rather than a silent 0
    if (threadIdx.x == 0) *dt_out = isinf(v) ? (double)NAN : cfl * h / fmax(v, 1.0);
  }
}

// Device address of g_noalloc_partial per device, looked up once per device
// (with that device current) and cached; the name itself is only a host-side
// stand-in and must never be handed to a kernel.  The cache entries are
// atomics: host threads making their first calls on one device at the same
// time may each look the address up, and all of them store the same value.
// A cudaDeviceReset unloads the module, after which a cached address is
// stale; the library's contexts do not survive a reset either.
static double* noalloc_scratch(int* st) {
  constexpr int kMaxDevices = 64;
  static std::atomic<double*> addr[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = HBF_ERR_CUDA;
    return nullptr;
  }
  double* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess || !p) {
      *st = HBF_ERR_CUDA;
      return nullptr;
    }
    a = (double*)p;
    addr[dev].store(a, std::memory_order_release);
  }
  *st = HBF_OK;
  return a;
}

// ---------------------------------------------------------------------------
// small elementwise kernels
// ---------------------------------------------------------------------------
template <typename TO, typename TI>
__global__ void k_convert(TO* __restrict__ out, const TI* __restrict__ in, long long n) {
  for_each4(
      n, aligned16_all(out, in),
      [&](long long q) {
        const V4<TI> a = ld4(in, q);
        st4(out, q, V4<TO>{{TO(a.v[0]), TO(a.v[1]), TO(a.v[2]), TO(a.v[3])}});
      },
      [&](long long e) { out[e] = TO(in[e]); });
}

// x (FP64) += e (FP32): the defect-correction update
__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ e, long long n) {
  for_each4(
      n, aligned16_all(x, e),
      [&](long long q) {
        V4<double> a = ld4(x, q);
        const V4<float> d = ld4(e, q);
#pragma unroll
        for (int i = 0; i < 4; ++i) a.v[i] += (double)d.v[i];
        st4(x, q, a);
      },
      [&](long long i) { x[i] += (double)e[i]; });
}

// p = r + beta (p - omega v)
template <typename T>
__global__ void k_bicg_p(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ v, T beta, T omega,
                         long long n) {
  for_each4(
      n, aligned16_all(p, r, v),
      [&](long long q) {
        V4<T> a = ld4(p, q);
        const V4<T> b = ld4(r, q), c = ld4(v, q);
#pragma unroll
        for (int i = 0; i < 4; ++i) a.v[i] = b.v[i] + beta * (a.v[i] - omega * c.v[i]);
        st4(p, q, a);
      },
      [&](long long e) { p[e] = r[e] + beta * (p[e] - omega * v[e]); });
}

// out = x - a y
template <typename T>
__global__ void k_axmy(T* __restrict__ out, const T* __restrict__ x, T a, const T* __restrict__ y, long long n) {
  for_each4(
      n, aligned16_all(out, x, y),
      [&](long long q) {
        const V4<T> b = ld4(x, q), c = ld4(y, q);
        V4<T> o;
#pragma unroll
        for (int i = 0; i < 4; ++i) o.v[i] = b.v[i] - a * c.v[i];
        st4(out, q, o);
      },
      [&](long long e) { out[e] = x[e] - a * y[e]; });
}

// x = x + alpha ph + omega sh
template <typename T>
__global__ void k_bicg_x(T* __restrict__ x, const T* __restrict__ ph, const T* __restrict__ sh, T alpha, T omega,
                         long long n) {
  for_each4(
      n, aligned16_all(x, ph, sh),
      [&](long long q) {
        V4<T> a = ld4(x, q);
        const V4<T> b = ld4(ph, q), c = ld4(sh, q);
#pragma unroll
        for (int i = 0; i < 4; ++i) a.v[i] = a.v[i] + alpha * b.v[i] + omega * c.v[i];
        st4(x, q, a);
      },
      [&](long long e) { x[e] = x[e] + alpha * ph[e] + omega * sh[e]; });
}

// sum of a*b over float arrays: FP32 products summed in FP32 over runs of
// kDotRun elements per thread, the runs summed in FP64 (GB300's FP64 rate is a
// small fraction of its FP32 rate, so a per-element FP64 product is the
// bottleneck of this reduction)
constexpr int kDotRun = 64;
__global__ void k_dot_partial_f(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                double* __restrict__ part) {
  double acc = 0.0;
  float run = 0.f;
  int k = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    run = fmaf(a[t], b[t], run);
    if (++k == kDotRun) {
      acc += (double)run;
      run = 0.f;
      k = 0;
    }
  }
  acc += (double)run;
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// max |x| over a float array (non-finite -> +inf)
__global__ void k_maxabs_partial_f(const float* __restrict__ x, long long n, double* __restrict__ part) {
  float m = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    float a = fabsf(x[t]);
    if (!isfinite(a)) a = INFINITY;
    m = fmaxf(m, a);
  }
  double acc = (double)m;
  __shared__ double sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

// the FP32 partials with 16-byte loads: products summed in FP32 over runs of
// kDotRun elements (kDotRun / 4 vectors), the runs in FP64; same order rules
// as k_reduce_partial_v.  A thread takes its vectors q0, q0 + T, ... one run
// at a time (nested loops, so that a run's loads are issued together); a run
// is added to the FP64 sum once it holds kDotRun / 4 vectors, and the last,
// shorter one (with thread 0's tail past the last whole vector) at the end.
constexpr int kRunVec = kDotRun / 4;

// acc, run: the thread's FP64 sum of finished runs and its open FP32 run;
// term(q, run) adds vector q's products to run
template <typename F>
__device__ __forceinline__ void dot_runs(long long tid, long long T, long long n4, double& acc, float& run, F term) {
  for (long long q0 = tid; q0 < n4; q0 += (long long)kRunVec * T) {
#pragma unroll 4
    for (int k = 0; k < kRunVec; ++k) {
      const long long q = q0 + (long long)k * T;
      if (q < n4) run = term(q, run);
    }
    if (q0 + (long long)(kRunVec - 1) * T < n4) {
      acc += (double)run;
      run = 0.f;
    }
  }
}

__device__ __forceinline__ float dot4(const float4& x, const float4& y, float run) {
  run = fmaf(x.x, y.x, run);
  run = fmaf(x.y, y.y, run);
  run = fmaf(x.z, y.z, run);
  return fmaf(x.w, y.w, run);
}

__device__ __forceinline__ void max_abs(float& m, float v) {
  float a = fabsf(v);
  if (!isfinite(a)) a = INFINITY;
  m = fmaxf(m, a);
}

__global__ void k_dot_partial_f4(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                 double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n >> 2;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  double acc = 0.0;
  float run = 0.f;
  dot_runs(tid, T, n4, acc, run, [&](long long q, float r) { return dot4(a4[q], b4[q], r); });
  if (tid == 0)
    for (long long e = n4 << 2; e < n; ++e) run = fmaf(a[e], b[e], run);
  acc += (double)run;
  block_partial<1>(acc, part);
}

// x.x and x.y in one pass over x (BiCGStab's t.t and t.s): partials of the
// first in part[0, gridDim), of the second in part[gridDim, 2 gridDim)
__global__ void k_dot2_partial_f4(const float* __restrict__ x, const float* __restrict__ y, long long n,
                                  double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n >> 2;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  double axx = 0.0, axy = 0.0;
  float rxx = 0.f, rxy = 0.f;
  for (long long q0 = tid; q0 < n4; q0 += (long long)kRunVec * T) {
#pragma unroll 4
    for (int k = 0; k < kRunVec; ++k) {
      const long long q = q0 + (long long)k * T;
      if (q < n4) {
        const float4 u = x4[q], v = y4[q];
        rxx = dot4(u, u, rxx);
        rxy = dot4(u, v, rxy);
      }
    }
    if (q0 + (long long)(kRunVec - 1) * T < n4) {
      axx += (double)rxx;
      axy += (double)rxy;
      rxx = rxy = 0.f;
    }
  }
  if (tid == 0)
    for (long long e = n4 << 2; e < n; ++e) {
      rxx = fmaf(x[e], x[e], rxx);
      rxy = fmaf(x[e], y[e], rxy);
    }
  block_partial<1>(axx + (double)rxx, part);
  __syncthreads();
  block_partial<1>(axy + (double)rxy, part + gridDim.x);
}

// out = x - a y (BiCGStab's r = s - omega t) with max |out| (non-finite ->
// +inf) and w.out (the next iteration's r^.r) in the same pass: partials of
// the max in part[0, gridDim), of the dot in part[gridDim, 2 gridDim)
__global__ void k_axmy_red_f4(float* __restrict__ out, const float* __restrict__ x, float a,
                              const float* __restrict__ y, const float* __restrict__ w, long long n,
                              double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n >> 2;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  const float4* w4 = reinterpret_cast<const float4*>(w);
  float4* o4 = reinterpret_cast<float4*>(out);
  double acc = 0.0;
  float run = 0.f, m = 0.f;
  dot_runs(tid, T, n4, acc, run, [&](long long q, float r) {
    const float4 u = x4[q], v = y4[q];
    float4 o;
    o.x = u.x - a * v.x;
    o.y = u.y - a * v.y;
    o.z = u.z - a * v.z;
    o.w = u.w - a * v.w;
    o4[q] = o;
    max_abs(m, o.x);
    max_abs(m, o.y);
    max_abs(m, o.z);
    max_abs(m, o.w);
    return dot4(w4[q], o, r);
  });
  if (tid == 0)
    for (long long e = n4 << 2; e < n; ++e) {
      const float o = x[e] - a * y[e];
      out[e] = o;
      max_abs(m, o);
      run = fmaf(w[e], o, run);
    }
  block_partial<0>((double)m, part);
  __syncthreads();
  block_partial<1>(acc + (double)run, part + gridDim.x);
}

__global__ void k_maxabs_partial_f4(const float* __restrict__ x, long long n, double* __restrict__ part) {
  const long long T = (long long)gridDim.x * blockDim.x, tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n >> 2;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  float m = 0.f;
#pragma unroll 4
  for (long long q = tid; q < n4; q += T) {
    const float4 v = x4[q];
    max_abs(m, v.x);
    max_abs(m, v.y);
    max_abs(m, v.z);
    max_abs(m, v.w);
  }
  if (tid == 0)
    for (long long e = n4 << 2; e < n; ++e) max_abs(m, x[e]);
  block_partial<0>((double)m, part);
}

// the two finals of a two-result partial kernel: block 0 reduces
// part[0, nb) with MODE0 into out[0], block 1 part[nb, 2 nb) with MODE1 into
// out[1]
template <int MODE0, int MODE1>
__global__ void k_reduce_final2(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  const int mode = blockIdx.x == 0 ? MODE0 : MODE1;
  const double* p = part + (size_t)blockIdx.x * nb;
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc = mode == 0 ? fmax(acc, p[t]) : acc + p[t];
  for (int off = 16; off > 0; off >>= 1) {
    double o = __shfl_xor_sync(0xffffffffu, acc, off);
    acc = mode == 0 ? fmax(acc, o) : acc + o;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = mode == 0 ? fmax(v, o) : v + o;
    }
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

static double reduce_dot_f(hbf_ctx* c, const float* a, const float* b, long long n, int* st) {
  if (aligned16(a) && aligned16(b))
    launch(c, kSlotReduce, k_dot_partial_f4, kRedBlocks, kThreads, a, b, n, c->partial);
  else
    launch(c, kSlotReduce, k_dot_partial_f, kRedBlocks, kThreads, a, b, n, c->partial);
  launch(c, kSlotReduce, k_reduce_final<1>, 1, 1024, (const double*)c->partial, kRedBlocks, c->dres);
  *st = cuda_check(c, cudaGetLastError(), "dot");
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

// both results of a two-result partial kernel (out[0], out[1]), one read
static int read_results2(hbf_ctx* c, double* r0, double* r1) {
  launch(c, kSlotReduce, k_reduce_final2<0, 1>, 2, 1024, (const double*)c->partial, kRedBlocks, c->dres);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->hres, c->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "reading a reduction");
  *r0 = c->hres[0];
  *r1 = c->hres[1];
  return HBF_OK;
}

// (x.x, x.y) in one pass; sum-sum finals
static int reduce_dot2_f(hbf_ctx* c, const float* x, const float* y, long long n, double* xx, double* xy) {
  launch(c, kSlotReduce, k_dot2_partial_f4, kRedBlocks, kThreads, x, y, n, c->partial);
  launch(c, kSlotReduce, k_reduce_final2<1, 1>, 2, 1024, (const double*)c->partial, kRedBlocks, c->dres);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->hres, c->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "reading a reduction");
  *xx = c->hres[0];
  *xy = c->hres[1];
  return HBF_OK;
}

static double reduce_max_abs_f(hbf_ctx* c, const float* x, long long n, int* st) {
  if (aligned16(x))
    launch(c, kSlotReduce, k_maxabs_partial_f4, kRedBlocks, kThreads, x, n, c->partial);
  else
    launch(c, kSlotReduce, k_maxabs_partial_f, kRedBlocks, kThreads, x, n, c->partial);
  launch(c, kSlotReduce, k_reduce_final<0>, 1, 1024, (const double*)c->partial, kRedBlocks, c->dres);
  *st = cuda_check(c, cudaGetLastError(), "max");
  if (*st) return NAN;
  return read_result(c, c->dres, st);
}

// threads of the single-block coarsest-level solver: enough for the largest
// colour class, in whole warps (fewer threads make each barrier cheaper)
static inline int bottom_threads(int colour_count) {
  int t = ((colour_count + 31) / 32) * 32;
  return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

// ---------------------------------------------------------------------------
// per-precision views of a level's arrays
// ---------------------------------------------------------------------------
template <typename T>
struct View;
template <>
struct View<double> {
  static double* vx(Level& L) { return L.vx; }
  static double* vb(Level& L) { return L.vb; }
  static double* vr(Level& L) { return L.vr; }
  static double* ef(Level& L, int a) { return L.ef[a]; }
  static double* cx(Level& L) { return L.cx; }
  static double* cb(Level& L) { return L.cb; }
  static double* cr(Level& L) { return L.cr; }
  static double* nx(Level& L) { return L.nx; }
  static double* nb(Level& L) { return L.nb; }
  static double* nr(Level& L) { return L.nr; }
};
template <>
struct View<float> {
  static float* vx(Level& L) { return L.fvx; }
  static float* vb(Level& L) { return L.fvb; }
  static float* vr(Level& L) { return L.fvr; }
  static float* ef(Level& L, int a) { return L.fef[a]; }
  static float* cx(Level& L) { return L.fcx; }
  static float* cb(Level& L) { return L.fcb; }
  static float* cr(Level& L) { return L.fcr; }
  static float* nx(Level& L) { return L.fnx; }
  static float* nb(Level& L) { return L.fnb; }
  static float* nr(Level& L) { return L.fnr; }
};

// ---------------------------------------------------------------------------
// problem interface for the generic driver
// ---------------------------------------------------------------------------
// One linear problem on the level hierarchy in arithmetic T.  hom0: level 0
// carries homogeneous boundary values (the error equation of the mixed
// solve); coarse levels are always homogeneous.
template <typename T>
struct Problem {
  hbf_ctx* c;
  int nlev;
  bool singular;
  bool hom0;
  Problem(hbf_ctx* ctx, bool sing, bool h0) : c(ctx), nlev((int)ctx->lv.size()), singular(sing), hom0(h0) {}
  virtual ~Problem() {}
  bool hom(int l) const { return l > 0 || hom0; }
  virtual T* x(int l) = 0;
  virtual T* b(int l) = 0;
  virtual T* r(int l) = 0;
  virtual long long count(int l) = 0;
  virtual void smooth(int l) = 0;
  // count sweeps (a problem may fuse or pipeline them)
  virtual void smooth_n(int l, int count) {
    for (int s = 0; s < count; ++s) smooth(l);
  }
  virtual void resid(int l) = 0;
  virtual void restrict_to(int l) = 0;  // b(l+1) = R r(l), x(l+1) = 0
  virtual void prolong_add(int l) = 0;  // x(l) += P x(l+1)
  virtual void bottom(int l) = 0;       // FP64 solve on the coarsest level
  virtual int sub_mean(int l, double* v) { (void)l; (void)v; return 0; }
  virtual int kind() const = 0;         // 0 viscous, 1 MAC, 2 nodal
  virtual double dense_beta() const { return 0.0; }
  // levels l..coarsest in one fused launch (hb_vcycle_tail.cuh); false when
  // l is not the context's tail level
  virtual bool tail(int l) { (void)l; return false; }
};

// dense inverse of the bottom operator of problem kind `kind` at level l
template <int D>
static void build_dense(hbf_ctx* c, int kind, int l, long long n, double beta) {
  Level& L = c->lv[l];
  Dense& Dn = c->dense[kind];
  const int m = kind == 0 ? (int)n : (int)n + 1;
  launch(c, kSlotBottom, k_dense_build<D>, (int)n, 128, kind, c->dX, c->dM, (int)n, m, (const double*)L.ef[0],
         (const double*)L.ef[1], (const double*)L.ef[2], L.g, beta);
  launch(c, kSlotBottom, k_gauss_jordan, 1, 256, (const double*)c->dM, m, c->dA, Dn.Minv);
  Dn.n = m;
  Dn.valid = true;
}

// coarsest level in FP64 for either precision (the FP32 path converts in and
// out): exact dense solve when it has at most kDenseMax unknowns, else
// nu_bottom smoothing sweeps
template <int D, typename T>
static void bottom_fp64(Problem<T>& P, int l, double* xd, double* bd, void (*run)(Problem<T>&, int, double*, double*)) {
  hbf_ctx* c = P.c;
  long long n = P.count(l);
  if (!std::is_same<T, double>::value) {
    launch(c, kSlotTransfer, k_convert<double, T>, grid_for(n), kThreads, bd, (const T*)P.b(l), n);
    launch(c, kSlotTransfer, k_zero<double>, grid_for(n), kThreads, xd, n);
  }
  if (P.singular) P.sub_mean(l, bd);
  if (n <= kDenseMax) {
    Dense& Dn = c->dense[P.kind()];
    if (!Dn.valid) build_dense<D>(c, P.kind(), l, n, P.dense_beta());
    launch(c, kSlotBottom, k_dense_apply, 1, 256, (const double*)Dn.Minv, Dn.n, (const double*)bd, (int)n, xd);
  } else {
    run(P, l, xd, bd);
  }
  if (P.singular) P.sub_mean(l, xd);
  if (!std::is_same<T, double>::value)
    launch(c, kSlotTransfer, k_convert<T, double>, grid_for(n), kThreads, P.x(l), (const double*)xd, n);
}

// ---------------------------------------------------------------------------
// fused tail of the V-cycle (k_vcycle_tail): from the first level with at
// most c->tail_cells cells (hbf_set_tail) down to the exact bottom solve and
// back in one launch of one block, instead of about twenty launches per level
// ---------------------------------------------------------------------------

static int tail_level(hbf_ctx* c) {
  if (c->tail_lf >= 0) return c->tail_lf;
  const int nl = (int)c->lv.size();
  const Geom& gb = c->lv[nl - 1].g;
  const bool dense = (long long)c->dim * gb.ncell <= kDenseMax && gb.nnode <= kDenseMax;
  int lf = nl;
  if (dense)
    for (int l = 1; l < nl; ++l)
      if (c->lv[l].g.ncell <= c->tail_cells) {
        lf = l;
        break;
      }
  c->tail_lf = lf;
  return lf;
}

template <typename T, typename A>
struct TailBlock {
  A lv[batch::kMaxLev];
  batch::XferArg<T> re[batch::kMaxLev];
  batch::XferArg<T> pr[batch::kMaxLev];
  batch::BottomArg<T> bot;
};

template <int D, typename T, int KIND>
static bool run_tail(hbf_ctx* c, int l, double beta) {
  using namespace batch;
  const int lf = tail_level(c);
  const int nl = (int)c->lv.size(), L = nl - 1;
  if (l != lf || lf >= nl || nl > kMaxLev) return false;
  const int pi = sizeof(T) == 4 ? 1 : 0;
  using A = typename std::conditional<KIND == kVisc, ViscArg<T>, PoisArg<T>>::type;
  using TB = TailBlock<T, A>;
  std::vector<unsigned char>& host = c->tail_host[KIND][pi];
  void*& dev = c->tail_dev[KIND][pi];
  const bool fresh = host.empty();
  if (fresh) {
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(TB)) != cudaSuccess) return false;  // fall back to level-by-level
    c->allocs.push_back(d);
    dev = d;
    host.assign(sizeof(TB), 0);
  }
  if (fresh || (KIND == kVisc && c->tail_beta[pi] != beta)) {
    TB* h = (TB*)host.data();
    auto X = [&](Level& Lv) -> T* { return KIND == kVisc ? View<T>::vx(Lv) : KIND == kMac ? View<T>::cx(Lv) : View<T>::nx(Lv); };
    auto Bv = [&](Level& Lv) -> T* { return KIND == kVisc ? View<T>::vb(Lv) : KIND == kMac ? View<T>::cb(Lv) : View<T>::nb(Lv); };
    auto R = [&](Level& Lv) -> T* { return KIND == kVisc ? View<T>::vr(Lv) : KIND == kMac ? View<T>::cr(Lv) : View<T>::nr(Lv); };
    const int ncomp = KIND == kVisc ? D : 1, sign = KIND == kVisc ? -1 : 1;
    for (int q = lf; q <= L; ++q) {
      Level& Lv = c->lv[q];
      A a;
      std::memset(&a, 0, sizeof a);
      a.x = X(Lv);
      a.b = Bv(Lv);
      a.g = Lv.g;
      if constexpr (KIND == kVisc) {
        a.out = R(Lv);
        for (int d = 0; d < D; ++d) a.ef[d] = View<T>::ef(Lv, d);
        a.beta = (T)beta;
        a.hom = 1;
      } else {
        a.r = R(Lv);
      }
      h->lv[q] = a;
      if (q < L) {
        Level& Cv = c->lv[q + 1];
        h->re[q] = XferArg<T>{R(Lv), Bv(Cv), X(Cv), Lv.g, Cv.g, ncomp, sign};
        h->pr[q] = XferArg<T>{X(Cv), X(Lv), nullptr, Lv.g, Cv.g, ncomp, sign};
      }
    }
    BottomArg<T> bt;
    std::memset(&bt, 0, sizeof bt);
    const Geom& gb = c->lv[L].g;
    bt.n = KIND == kVisc ? D * gb.ncell : KIND == kMac ? gb.ncell : gb.nnode;
    bt.m = KIND == kVisc ? bt.n : bt.n + 1;
    bt.Minv = c->dense[KIND].Minv;
    bt.x = X(c->lv[L]);
    bt.b = Bv(c->lv[L]);
    bt.g = gb;
    bt.kind = KIND;
    bt.level = L;
    h->bot = bt;
    // pageable source: the call returns once the bytes are staged
    if (cudaMemcpyAsync(dev, h, sizeof(TB), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) return false;
    if (KIND == kVisc) c->tail_beta[pi] = beta;
  }
  ensure_dense(c, KIND, beta);  // the viscous inverse changes with eta and dt
  TB* d = (TB*)dev;
  TailTabs tb;
  for (int q = 0; q < kMaxLev; ++q) {
    tb.lv[q] = &d->lv[q];
    tb.re[q] = &d->re[q];
    tb.pr[q] = &d->pr[q];
  }
  tb.bot = &d->bot;
  if (any_per(c->g))
    launch(c, kSlotCoarse, k_vcycle_tail<D, T, KIND, true>, 1, kThreads, tb, lf, 1, (const int*)nullptr, c->cfg.nu1,
           c->cfg.nu2);
  else
    launch(c, kSlotCoarse, k_vcycle_tail<D, T, KIND, false>, 1, kThreads, tb, lf, 1, (const int*)nullptr, c->cfg.nu1,
           c->cfg.nu2);
  return true;
}

static bool staged_op(hbf_ctx* c, int slot, const float* u, const float* b, float* out, const float* eta,
                      const Geom& g, float beta, int hm);

template <int D, typename T>
struct ViscProblem : Problem<T> {
  using Problem<T>::c;
  T* x0;
  const T* b0 = nullptr;  // level-0 right-hand side in place of the level's own array (read only)
  double beta;
  const bool sp;  // level 0 in the colour-split layout (FP32 only)
  ViscProblem(hbf_ctx* ctx, T* x_in, double bt, bool h0)
      : Problem<T>(ctx, false, h0), x0(x_in), beta(bt), sp(sizeof(T) == 4 && D == 3 && split0(ctx)) {}
  int kind() const override { return 0; }
  double dense_beta() const override { return beta; }
  bool tail(int l) override { return run_tail<D, T, batch::kVisc>(c, l, beta); }
  T* x(int l) override { return l == 0 ? x0 : View<T>::vx(c->lv[l]); }
  T* b(int l) override { return (l == 0 && b0) ? const_cast<T*>(b0) : View<T>::vb(c->lv[l]); }
  T* r(int l) override { return View<T>::vr(c->lv[l]); }
  long long count(int l) override { return (long long)D * c->lv[l].g.ncell; }
  void smooth(int l) override {
    Level& L = c->lv[l];
    const int slot = l == 0 ? kSlotViscSmooth : kSlotCoarse;
    const dim3 blk(kThreads, 1, 1);
    const dim3 grd((unsigned)grid_for(rbx_count<D>(L.g), 152 * 24), 1, 1);
    const int hm = (int)this->hom(l);
    if (l == 0 && sp) {
      if constexpr (D == 3 && sizeof(T) == 4) {
        const float* e0 = (const float*)L.feta;
        const dim3 sg = split_sweep_grid(L.g), sb = split_sweep_block(L.g);
        // pairs read by 8-byte loads: even rows (n0 / 2) and 8-byte aligned arrays
        const bool vec = (L.g.n[0] / 2) % 2 == 0 && aligned8(x(l)) && aligned8(b(l)) && aligned8(e0);
        for (int col = 0; col < 2; ++col)
          vec ? launch3(c, slot, k_visc_smooth_split<0, true>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm)
              : launch3(c, slot, k_visc_smooth_split<0, false>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm);
        for (int col = 0; col < 2; ++col)
          vec ? launch3(c, slot, k_visc_smooth_split<1, true>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm)
              : launch3(c, slot, k_visc_smooth_split<1, false>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm);
        for (int col = 0; col < 2; ++col)
          vec ? launch3(c, slot, k_visc_smooth_split<2, true>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm)
              : launch3(c, slot, k_visc_smooth_split<2, false>, sg, sb, x(l), (const T*)b(l), e0, L.g, col, (T)beta, hm);
      }
      return;
    }
    if (cell_eta(l) && staged_sweeps(l, hm)) return;
    if (cell_eta(l)) {
      // FP32 finest level: face viscosities from the cell viscosity
      const T* e0 = (const T*)L.feta;
      for (int col = 0; col < 2; ++col)
        if (any_per(c->g))
          launch3(c, slot, k_visc_smooth_c<D, T, 0, true, true>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                (T)beta, hm);
        else
          launch3(c, slot, k_visc_smooth_c<D, T, 0, true, false>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                (T)beta, hm);
      for (int col = 0; col < 2; ++col)
        if (any_per(c->g))
          launch3(c, slot, k_visc_smooth_c<D, T, 1, true, true>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                (T)beta, hm);
        else
          launch3(c, slot, k_visc_smooth_c<D, T, 1, true, false>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                (T)beta, hm);
      if (D == 3)
        for (int col = 0; col < 2; ++col)
          if (any_per(c->g))
            launch3(c, slot, k_visc_smooth_c<D, T, 2, true, true>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                  (T)beta, hm);
          else
            launch3(c, slot, k_visc_smooth_c<D, T, 2, true, false>, grd, blk, x(l), (const T*)b(l), e0, e0, e0, L.g, col,
                  (T)beta, hm);
      return;
    }
    const T* e0 = View<T>::ef(L, 0);
    const T* e1 = View<T>::ef(L, 1);
    const T* e2 = View<T>::ef(L, 2);
    for (int col = 0; col < 2; ++col)
      if (any_per(c->g))
        launch3(c, slot, k_visc_smooth_c<D, T, 0, false, true>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta, hm);
      else
        launch3(c, slot, k_visc_smooth_c<D, T, 0, false, false>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta, hm);
    for (int col = 0; col < 2; ++col)
      if (any_per(c->g))
        launch3(c, slot, k_visc_smooth_c<D, T, 1, false, true>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta, hm);
      else
        launch3(c, slot, k_visc_smooth_c<D, T, 1, false, false>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta, hm);
    if (D == 3)
      for (int col = 0; col < 2; ++col)
        if (any_per(c->g))
          launch3(c, slot, k_visc_smooth_c<D, T, 2, false, true>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta,
                hm);
        else
          launch3(c, slot, k_visc_smooth_c<D, T, 2, false, false>, grd, blk, x(l), (const T*)b(l), e0, e1, e2, L.g, col, (T)beta,
                hm);
  }
  // the FP32 finest level forms its face viscosities from the cell viscosity
  bool cell_eta(int l) const { return l == 0 && sizeof(T) == 4 && c->lv[0].feta != nullptr; }
  // 3D FP32 finest level with walls on every axis: the sweeps of k_visc_smooth_c
  // with the planes staged in shared memory by TMA (hb_visc_tma.cuh); false
  // (nothing launched) when the staged sweep is off or the level does not
  // meet its layout rules
  bool staged_sweeps(int l, int hm);
  // 3D FP32 finest level: each component's red-black sweep in one launch
  // (hb_visc_fused.cuh), alternating between x and the level's second array
  void smooth_n(int l, int count) override {
    const bool walls = !c->g.per[0] && !c->g.per[1] && !c->g.per[2];
    if (!(D == 3 && cell_eta(l) && c->fused_sweep && c->lv[0].fvx2 && walls)) {
      Problem<T>::smooth_n(l, count);
      return;
    }
    fused_sweeps(l, count);
  }
  void fused_sweeps(int l, int count);
  void resid(int l) override {
    Level& L = c->lv[l];
    const dim3 blk(256, 1, 1);
    const dim3 grd(op3_blocks<D>(L.g), 1, 1);
    if (l == 0 && sp) {
      if constexpr (D == 3 && sizeof(T) == 4)
        launch3(c, kSlotViscResid, k_visc_op_split, split_grid(L.g), split_block_dim(L.g, 2), (const T*)x(l),
                (const T*)b(l), r(l), (const T*)L.feta, L.g, (T)beta, (int)this->hom(l));
      return;
    }
    if (cell_eta(l)) {
      const T* e0 = (const T*)L.feta;
      if constexpr (std::is_same<T, float>::value)
        if (staged_op(c, kSlotViscResid, x(l), b(l), r(l), L.feta, L.g, (float)beta, (int)this->hom(l))) return;
      if (any_per(c->g))
        launch3(c, kSlotViscResid, k_visc_op3<D, T, true, true>, grd, blk, (const T*)x(l), (const T*)b(l), r(l), e0, e0, e0,
              L.g, (T)beta, (int)this->hom(l));
      else
        launch3(c, kSlotViscResid, k_visc_op3<D, T, true, false>, grd, blk, (const T*)x(l), (const T*)b(l), r(l), e0, e0, e0,
              L.g, (T)beta, (int)this->hom(l));
      return;
    }
    if (any_per(c->g))
      launch3(c, l == 0 ? kSlotViscResid : kSlotCoarse, k_visc_op3<D, T, false, true>, grd, blk, (const T*)x(l), (const T*)b(l), r(l),
            (const T*)View<T>::ef(L, 0), (const T*)View<T>::ef(L, 1), (const T*)View<T>::ef(L, 2), L.g, (T)beta,
            (int)this->hom(l));
    else
      launch3(c, l == 0 ? kSlotViscResid : kSlotCoarse, k_visc_op3<D, T, false, false>, grd, blk, (const T*)x(l), (const T*)b(l), r(l),
            (const T*)View<T>::ef(L, 0), (const T*)View<T>::ef(L, 1), (const T*)View<T>::ef(L, 2), L.g, (T)beta,
            (int)this->hom(l));
  }
  void restrict_to(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    long long n = (long long)D * C.g.ncell;
    if (l == 0 && sp)
      launch(c, kSlotTransfer, k_restrict_cells<D, T, true>, grid_for(n), kThreads, r(l), b(l + 1), F.g, C.g, D);
    else
      launch(c, kSlotTransfer, k_restrict_cells<D, T>, grid_for(n), kThreads, r(l), b(l + 1), F.g, C.g, D);
    launch(c, kSlotTransfer, k_zero<T>, grid_for(n), kThreads, x(l + 1), n);
  }
  void prolong_add(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    if (l == 0 && sp) {
      launch(c, kSlotTransfer, k_prolong_cells_add_c<D, T, false, true>, grid_for((long long)D * C.g.ncell), kThreads, x(l),
             x(l + 1), F.g, C.g, D, T(-1));
    } else {
      if (any_per(c->g))
        launch(c, kSlotTransfer, k_prolong_cells_add_c<D, T, true>, grid_for((long long)D * C.g.ncell), kThreads, x(l), x(l + 1),
           F.g, C.g, D, T(-1));
      else
        launch(c, kSlotTransfer, k_prolong_cells_add_c<D, T, false>, grid_for((long long)D * C.g.ncell), kThreads, x(l), x(l + 1),
           F.g, C.g, D, T(-1));
    }
  }
  static void run_bottom(Problem<T>& P, int l, double* xd, double* bd) {
    auto& S = static_cast<ViscProblem&>(P);
    Level& L = S.c->lv[l];
    launch(S.c, kSlotBottom, k_visc_bottom<D, double>, 1, bottom_threads(rb_count<D>(L.g)), xd, (const double*)bd, (const double*)L.ef[0],
           (const double*)L.ef[1], (const double*)L.ef[2], L.g, S.beta, S.c->cfg.nu_bottom, (int)S.hom(l));
  }
  void bottom(int l) override {
    Level& L = c->lv[l];
    double* xd = std::is_same<T, double>::value ? (double*)x(l) : L.vx;
    double* bd = std::is_same<T, double>::value ? (double*)b(l) : L.vb;
    bottom_fp64<D, T>(*this, l, xd, bd, &run_bottom);
  }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point, so that
// the library links against the runtime only
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tiled FP32 map of a cell array of level geometry g: rank 3 (n0, n1, n2), or
// rank 4 with ncomp component arrays of ncell cells each.  Box bx x by x 1
// (x bc components); coordinates outside the grid read zeros.  Needs
// n0 % 4 == 0 (row strides in multiples of 16 bytes) and a 16-byte aligned
// base.
static bool encode_cells(CUtensorMap* m, const void* base, const Geom& g, int ncomp, int bx, int by, int bc) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)base & 15) || g.n[0] % 4) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)ncomp};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4, (cuuint64_t)g.ncell * 4};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bc};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ncomp > 0 ? 4 : 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One colour sweep of every component, staged: tile TX x TY, ring of NS stages
template <int TX, int TY, int NS>
static bool staged_launches(hbf_ctx* c, int slot, float* u, const float* b, const float* eta, const Geom& g, float beta,
                            int hm, int tz) {
  using Lay = tma::Layout<TX, TY>;
  CUtensorMap mu, me, mb;
  if (!encode_cells(&mu, u, g, 3, Lay::PX, Lay::PY, 3) || !encode_cells(&me, eta, g, 0, Lay::PX, Lay::PY, 1) ||
      !encode_cells(&mb, b, g, 3, TX, TY, 1))
    return false;
  void (*kern[3])(const CUtensorMap, const CUtensorMap, const CUtensorMap, float*, const float*, const float*,
                  const Geom, const tma::SweepGrid, int, float, int, int*) = {
      tma::k_visc_smooth_tma<0, TX, TY, NS>, tma::k_visc_smooth_tma<1, TX, TY, NS>,
      tma::k_visc_smooth_tma<2, TX, TY, NS>};
  static std::atomic<bool> attr{false};
  const int smem = Lay::smem(NS);
  if (!attr.load()) {
    for (auto k : kern)
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
    attr.store(true);
  }
  const tma::SweepGrid sg = tma::sweep_grid<TX, TY>(g, tz);
  const dim3 grd((unsigned)sg.blocks(), 1, 1), blk(tma::kThreads, 1, 1);
  for (int q = 0; q < 3; ++q)
    for (int col = 0; col < 2; ++col)
      launch_smem(c, slot, kern[q], grd, blk, (size_t)smem, mu, me, mb, u, b, eta, g, sg, col, beta, hm,
                  c->sweep_err);
  return true;
}

template <int D, typename T>
bool ViscProblem<D, T>::staged_sweeps(int l, int hm) {
  if constexpr (D == 3 && std::is_same<T, float>::value) {
    const Geom& g = c->lv[l].g;
    if (c->staged_tx == 0 || g.per[0] || g.per[1] || g.per[2] || !c->sweep_err) return false;
    float* u = x(l);
    const float* bb = b(l);
    const float* e = c->lv[l].feta;
    const int tz = c->staged_tz;
    if (c->staged_tx == 64) return staged_launches<64, 8, 6>(c, kSlotViscSmooth, u, bb, e, g, (float)beta, hm, tz);
    return staged_launches<128, 8, 4>(c, kSlotViscSmooth, u, bb, e, g, (float)beta, hm, tz);
  }
  (void)l;
  (void)hm;
  return false;
}

// u - beta L u (b == nullptr) or b - (u - beta L u) on the 3D FP32 finest
// level with the planes staged by TMA (hb_visc_tma.cuh): tile 64 x rows,
// ring of 4 stages; false (nothing launched) when the staged operator is off,
// an axis is periodic, or the arrays do not meet the layout rules
template <int TY>
static bool staged_op_launch(hbf_ctx* c, int slot, const float* u, const float* b, float* out, const float* eta,
                             const Geom& g, float beta, int hm) {
  constexpr int TX = 64, NS = 4;
  using Lay = tma::Layout<TX, TY, false>;
  CUtensorMap mu, me;
  if (!encode_cells(&mu, u, g, 3, Lay::PX, Lay::PY, 3) || !encode_cells(&me, eta, g, 0, Lay::PX, Lay::PY, 1))
    return false;
  auto kern = tma::k_visc_op_tma<TX, TY, NS>;
  static std::atomic<bool> attr{false};
  const int smem = Lay::smem(NS);
  if (!attr.load()) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
    attr.store(true);
  }
  const tma::SweepGrid sg = tma::sweep_grid<TX, TY>(g, c->staged_op_tz);
  launch_smem(c, slot, kern, dim3((unsigned)sg.blocks(), 1, 1), dim3(tma::kThreads, 1, 1), (size_t)smem, mu, me, u, b,
              out, eta, g, sg, beta, hm, c->sweep_err);
  return true;
}

static bool staged_op(hbf_ctx* c, int slot, const float* u, const float* b, float* out, const float* eta,
                      const Geom& g, float beta, int hm) {
  if (c->dim != 3 || c->staged_op_rows == 0 || any_per(g) || !c->sweep_err || !eta) return false;
  if (c->staged_op_rows == 4) return staged_op_launch<4>(c, slot, u, b, out, eta, g, beta, hm);
  return staged_op_launch<8>(c, slot, u, b, out, eta, g, beta, hm);
}

static int take_sweep_err(hbf_ctx* c) {
  if (!c->sweep_err || (c->staged_tx == 0 && c->staged_op_rows == 0)) return HBF_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->sweep_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "reading the sweep status");
  if (!h) return HBF_OK;
  cudaMemsetAsync(c->sweep_err, 0, sizeof(int), c->stream);
  return fail(c, HBF_ERR_TIMEOUT, "a staged viscous sweep gave up waiting for its loads");
}

template <int D, typename T>
void ViscProblem<D, T>::fused_sweeps(int l, int count) {
  if constexpr (D == 3 && std::is_same<T, float>::value) {
    Level& L = c->lv[l];
    const long long n = L.g.ncell;
    static bool attr[3] = {false, false, false};
    void (*kern[3])(const float*, const float*, const float*, const float*, const float*, float*, const Geom, float,
                    int) = {fused::k_visc_sweep_rb<0>, fused::k_visc_sweep_rb<1>, fused::k_visc_sweep_rb<2>};
    for (int q = 0; q < 3; ++q)
      if (!attr[q]) {
        cudaFuncSetAttribute(kern[q], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(fused::Smem));
        attr[q] = true;
      }
    T* home = x(l);
    T* cur = home;
    T* oth = L.fvx2;
    const T* bb = b(l);
    const float* e0 = L.feta;
    const int hm = (int)this->hom(l);
    const dim3 grd = fused::sweep_grid(L.g);
    for (int s = 0; s < count; ++s) {
      // component q reads the components before it from oth (already swept)
      // and those after it from cur
      for (int q = 0; q < 3; ++q) {
        const int a0 = q == 0 ? 1 : 0, a1 = q == 2 ? 1 : 2;
        const float* pa = (a0 < q ? oth : cur) + a0 * n;
        const float* pb = (a1 < q ? oth : cur) + a1 * n;
        launch_smem(c, kSlotViscSmooth, kern[q], grd, dim3(fused::NT), sizeof(fused::Smem), (const float*)cur + q * n,
                    pa, pb, e0, bb + q * n, oth + q * n, L.g, (float)beta, hm);
      }
      T* t = cur;
      cur = oth;
      oth = t;
    }
    if (cur != home)
      cudaMemcpyAsync(home, cur, (size_t)3 * n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  } else {
    Problem<T>::smooth_n(l, count);
  }
}

template <int D, typename T>
struct MacProblem : Problem<T> {
  using Problem<T>::c;
  T* x0;
  MacProblem(hbf_ctx* ctx, T* x_in) : Problem<T>(ctx, true, true), x0(x_in) {}
  int kind() const override { return 1; }
  bool tail(int l) override { return run_tail<D, T, batch::kMac>(c, l, 0.0); }
  T* x(int l) override { return l == 0 ? x0 : View<T>::cx(c->lv[l]); }
  T* b(int l) override { return View<T>::cb(c->lv[l]); }
  T* r(int l) override { return View<T>::cr(c->lv[l]); }
  long long count(int l) override { return c->lv[l].g.ncell; }
  void smooth(int l) override {
    Level& L = c->lv[l];
    int nb = grid_for(rb_count<D>(L.g));
    for (int col = 0; col < 2; ++col)
      {
        if (any_per(c->g))
          launch(c, l == 0 ? kSlotCellSmooth : kSlotCoarse, k_cell_smooth<D, T, true>, nb, kThreads, x(l), b(l), L.g, col);
        else
          launch(c, l == 0 ? kSlotCellSmooth : kSlotCoarse, k_cell_smooth<D, T, false>, nb, kThreads, x(l), b(l), L.g, col);
      }
  }
  void resid(int l) override {
    Level& L = c->lv[l];
    {
      if (any_per(c->g))
        launch(c, l == 0 ? kSlotCellResid : kSlotCoarse, k_cell_resid<D, T, true>, grid_for(L.g.ncell), kThreads, x(l), b(l),
           r(l), L.g);
      else
        launch(c, l == 0 ? kSlotCellResid : kSlotCoarse, k_cell_resid<D, T, false>, grid_for(L.g.ncell), kThreads, x(l), b(l),
           r(l), L.g);
    }
  }
  void restrict_to(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotTransfer, k_restrict_cells<D, T>, grid_for(C.g.ncell), kThreads, r(l), b(l + 1), F.g, C.g, 1);
    launch(c, kSlotTransfer, k_zero<T>, grid_for(C.g.ncell), kThreads, x(l + 1), (long long)C.g.ncell);
  }
  void prolong_add(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    {
      if (any_per(c->g))
        launch(c, kSlotTransfer, k_prolong_cells_add_c<D, T, true>, grid_for(C.g.ncell), kThreads, x(l), x(l + 1), F.g, C.g, 1,
           T(1));
      else
        launch(c, kSlotTransfer, k_prolong_cells_add_c<D, T, false>, grid_for(C.g.ncell), kThreads, x(l), x(l + 1), F.g, C.g, 1,
           T(1));
    }
  }
  static void run_bottom(Problem<T>& P, int l, double* xd, double* bd) {
    Level& L = P.c->lv[l];
    launch(P.c, kSlotBottom, k_cell_bottom<D, double>, 1, bottom_threads(rb_count<D>(L.g)), xd, (const double*)bd, L.g, P.c->cfg.nu_bottom);
  }
  void bottom(int l) override {
    Level& L = c->lv[l];
    double* xd = std::is_same<T, double>::value ? (double*)x(l) : L.cx;
    double* bd = std::is_same<T, double>::value ? (double*)b(l) : L.cb;
    bottom_fp64<D, T>(*this, l, xd, bd, &run_bottom);
  }
  int sub_mean(int l, double* v) override {
    Level& L = c->lv[l];
    int st = reduce_to_device<1>(c, v, L.g.ncell, c->dres + 1);
    if (st) return st;
    launch(c, kSlotTransfer, k_sub_mean<double>, grid_for(L.g.ncell), kThreads, v, (long long)L.g.ncell,
           (const double*)(c->dres + 1), 1.0 / (double)L.g.ncell);
    return cuda_check(c, cudaGetLastError(), "k_sub_mean");
  }
};

template <int D, typename T>
struct NodalProblem : Problem<T> {
  using Problem<T>::c;
  T* x0;
  NodalProblem(hbf_ctx* ctx, T* x_in) : Problem<T>(ctx, true, true), x0(x_in) {}
  int kind() const override { return 2; }
  bool tail(int l) override { return run_tail<D, T, batch::kNodal>(c, l, 0.0); }
  T* x(int l) override { return l == 0 ? x0 : View<T>::nx(c->lv[l]); }
  T* b(int l) override { return View<T>::nb(c->lv[l]); }
  T* r(int l) override { return View<T>::nr(c->lv[l]); }
  long long count(int l) override { return c->lv[l].g.nnode; }
  void smooth(int l) override {
    Level& L = c->lv[l];
    for (int col = 0; col < (1 << D); ++col)
      {
        if (any_per(c->g))
          launch(c, l == 0 ? kSlotNodalSmooth : kSlotCoarse, k_nodal_smooth<D, T, true>, grid_for(mc_count<D>(L.g, col)),
             kThreads, x(l), b(l), L.g, col);
        else
          launch(c, l == 0 ? kSlotNodalSmooth : kSlotCoarse, k_nodal_smooth<D, T, false>, grid_for(mc_count<D>(L.g, col)),
             kThreads, x(l), b(l), L.g, col);
      }
  }
  void resid(int l) override {
    Level& L = c->lv[l];
    {
      if (any_per(c->g))
        launch(c, l == 0 ? kSlotNodalResid : kSlotCoarse, k_nodal_resid<D, T, true>, grid_for(L.g.nnode), kThreads, x(l), b(l),
           r(l), L.g);
      else
        launch(c, l == 0 ? kSlotNodalResid : kSlotCoarse, k_nodal_resid<D, T, false>, grid_for(L.g.nnode), kThreads, x(l), b(l),
           r(l), L.g);
    }
  }
  void restrict_to(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    {
      if (any_per(c->g))
        launch(c, kSlotTransfer, k_restrict_nodes<D, T, true>, grid_for(C.g.nnode), kThreads, r(l), b(l + 1), F.g, C.g);
      else
        launch(c, kSlotTransfer, k_restrict_nodes<D, T, false>, grid_for(C.g.nnode), kThreads, r(l), b(l + 1), F.g, C.g);
    }
    launch(c, kSlotTransfer, k_zero<T>, grid_for(C.g.nnode), kThreads, x(l + 1), (long long)C.g.nnode);
  }
  void prolong_add(int l) override {
    Level &F = c->lv[l], &C = c->lv[l + 1];
    launch(c, kSlotTransfer, k_prolong_nodes_add<D, T>, grid_for(F.g.nnode), kThreads, x(l), x(l + 1), F.g, C.g);
  }
  static void run_bottom(Problem<T>& P, int l, double* xd, double* bd) {
    Level& L = P.c->lv[l];
    launch(P.c, kSlotBottom, k_nodal_bottom<D, double>, 1, bottom_threads(mc_count<D>(L.g, 0)), xd, (const double*)bd, L.g, P.c->cfg.nu_bottom);
  }
  void bottom(int l) override {
    Level& L = c->lv[l];
    double* xd = std::is_same<T, double>::value ? (double*)x(l) : L.nx;
    double* bd = std::is_same<T, double>::value ? (double*)b(l) : L.nb;
    bottom_fp64<D, T>(*this, l, xd, bd, &run_bottom);
  }
  int sub_mean(int l, double* v) override {
    Level& L = c->lv[l];
    Geom gsave = c->g;
    c->g = L.g;  // the weighted reduction reads the level geometry from the context
    int st = reduce_to_device<2>(c, v, L.g.nnode, c->dres + 1);
    c->g = gsave;
    if (st) return st;
    double wsum = (double)L.g.n[0] * L.g.n[1] * (D == 3 ? L.g.n[2] : 1);
    launch(c, kSlotTransfer, k_sub_mean<double>, grid_for(L.g.nnode), kThreads, v, (long long)L.g.nnode,
           (const double*)(c->dres + 1), 1.0 / wsum);
    return cuda_check(c, cudaGetLastError(), "k_sub_mean");
  }
};

template <typename T>
static void vcycle(Problem<T>& P, int l, const SolverCfg& cfg) {
  if (P.tail(l)) return;
  if (l == P.nlev - 1) {
    P.bottom(l);
    return;
  }
  P.smooth_n(l, cfg.nu1);
  P.resid(l);
  P.restrict_to(l);
  vcycle(P, l + 1, cfg);
  P.prolong_add(l);
  P.smooth_n(l, cfg.nu2);
}

static inline int l0slot() { return kSlotViscResid; }

static int finish(hbf_ctx* c, int cycles, double r0, double rn, double bnorm, double tol, hbf_solve_stats* out) {
  hbf_solve_stats s;
  s.cycles = cycles;
  s.r0 = r0;
  s.rnorm = rn;
  s.bnorm = bnorm;
  s.converged = rn <= tol;
  s.guess = 0;
  if (out) *out = s;
  if (!std::isfinite(rn) || !std::isfinite(bnorm)) return fail(c, HBF_ERR_NONFINITE, "non-finite residual norm");
  if (!s.converged) {
    char buf[160];
    snprintf(buf, sizeof buf, "multigrid did not converge: %d cycles, residual %.3e > tol %.3e", cycles, rn, tol);
    return fail(c, HBF_ERR_NOT_CONVERGED, buf);
  }
  return HBF_OK;
}

// Plain FP64 multigrid (P64 only) or FP64 defect correction around FP32
// V-cycles (P32 given): r = b - A x in FP64; solve A e = r by one FP32
// V-cycle from e = 0; x += e in FP64; repeat to the same FP64 tolerance.
static int mg_solve(Problem<double>& P, Problem<float>* P32, const double* b_in, hbf_solve_stats* out) {
  hbf_ctx* c = P.c;
  const SolverCfg& cfg = c->cfg;
  long long n0 = P.count(0);
  int st = cuda_check(c, cudaMemcpyAsync(P.b(0), b_in, n0 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream),
                      "copy rhs");
  if (st) return st;
  if (P.singular) {
    if ((st = P.sub_mean(0, P.b(0)))) return st;
    if ((st = P.sub_mean(0, P.x(0)))) return st;
  }
  double bnorm = reduce_max_abs(c, P.b(0), n0, &st);
  if (st) return st;
  P.resid(0);
  double rn = reduce_max_abs(c, P.r(0), n0, &st);
  if (st) return st;
  double r0 = rn;
  if (bnorm == 0.0) bnorm = rn;
  double tol = cfg.rtol * bnorm;
  int cycles = 0;
  while (rn > tol && cycles < cfg.max_cycles && std::isfinite(rn)) {
    if (P32) {
      launch(c, kSlotTransfer, k_convert<float, double>, grid_for(n0), kThreads, P32->b(0), (const double*)P.r(0), n0);
      launch(c, kSlotTransfer, k_zero<float>, grid_for(n0), kThreads, P32->x(0), n0);
      vcycle(*P32, 0, cfg);
      launch(c, kSlotTransfer, k_add_f32, grid_for(n0), kThreads, P.x(0), (const float*)P32->x(0), n0);
    } else {
      vcycle(P, 0, cfg);
    }
    ++cycles;
    if (P.singular && (st = P.sub_mean(0, P.x(0)))) return st;
    P.resid(0);
    rn = reduce_max_abs(c, P.r(0), n0, &st);
    if (st) return st;
  }
  if ((st = cuda_check(c, cudaGetLastError(), "multigrid kernels"))) return st;
  return finish(c, cycles, r0, rn, bnorm, tol, out);
}

// coarse-level face eta from the level-0 faces (and FP32 copies when mixed)
template <int D>
static void build_eta_levels(hbf_ctx* c) {
  for (size_t l = 1; l < c->lv.size(); ++l) {
    Level &F = c->lv[l - 1], &C = c->lv[l];
    for (int a = 0; a < D; ++a)
      launch(c, kSlotTransfer, k_restrict_faces<D, double>, grid_for(C.g.nface[a]), kThreads, (const double*)F.ef[a],
             C.ef[a], a, F.g, C.g);
  }
  if (c->precision == HBF_MIXED) {
    for (size_t l = 1; l < c->lv.size(); ++l) {
      Level& L = c->lv[l];
      for (int a = 0; a < D; ++a)
        launch(c, kSlotTransfer, k_convert<float, double>, grid_for(L.g.nface[a]), kThreads, L.fef[a],
               (const double*)L.ef[a], (long long)L.g.nface[a]);
    }
    // the finest level of the FP32 V-cycles reads the cell viscosity (the
    // level-0 faces are the means of its cells, wall faces the interior cell)
    Level& L0 = c->lv[0];
    if (split0(c))
      launch(c, kSlotTransfer, k_split_from, grid_for(L0.g.ncell / 2), kThreads, L0.feta, (const double*)c->eta,
             (const double*)nullptr, L0.g, 1);
    else
      launch(c, kSlotTransfer, k_convert<float, double>, grid_for(L0.g.ncell), kThreads, L0.feta,
             (const double*)c->eta, (long long)L0.g.ncell);
  }
}

// BiCGStab (van der Vorst 1992) on (I - beta L_eta) u = b, right-preconditioned
// by one V-cycle of the homogeneous operator from a zero guess (FP64, or FP32
// in mixed mode).  The V-cycle alone does not converge for every viscosity
// field of the regularised law; as a preconditioner it does.  Stops when the
// recursive residual meets the tolerance and the true FP64 residual confirms
// it; otherwise restarts from the true residual.  cycles = iterations.
// Mixed precision: FP64 defect correction (r = b - A x and x += e in FP64)
// around an FP32 BiCGStab on A e = r, itself preconditioned by FP32 V-cycles,
// run until its residual drops by inner_drop (or kInnerMax iterations).
// cycles = total inner iterations.
constexpr int kInnerMax = 40;  // the drop is c->inner_drop (hbf_set_inner_drop, default 1e-3)

// x (FP64) += a d (FP32);  r (FP64) -= a w (FP32)
__global__ void k_add_scaled_f32(double* __restrict__ x, double a, const float* __restrict__ d, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] += a * (double)d[t];
}

// y = x - y
__global__ void k_rsub(const double* __restrict__ x, double* y, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = x[t] - y[t];
}

// out (FP32) = a - b (FP64)
__global__ void k_diff_to_f32(float* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b,
                              long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = (float)(a[t] - b[t]);
}

// Initial guess of the mixed-precision viscous solve (not in the paper; the
// solve still runs to its FP64 tolerance).  From x = u^m with FP64 residual
// r = b - A x, minimal-residual steps along up to two directions d, each
// taken only if it lowers max |r|:
//   w = A_hom d (the FP32 operator, homogeneous walls: the operator of a
//   correction), alpha = (r, w) / (w, w), x += alpha d, r -= alpha w.
// The directions: the previous step's increment u*^{m-1} - u^{m-1} (mode 1;
// where Crank-Nicolson leaves stiff modes flipping sign, alpha comes out
// near -1), then the network's direction for the remaining residual
// (mode 2).  *used: bit 0 the increment, bit 1 the network.
template <int D>
static int visc_guess(hbf_ctx* c, double beta, double* x, double* r, double* rn, int* used) {
  const ProfRegion region(c, kSlotGuess);  // the whole section (regions do not nest)
  Level& L0 = c->lv[0];
  const long long n = (long long)D * L0.g.ncell;
  const int nb = grid_for(n);
  const float fbeta = (float)beta;
  int st = 0;
  float* cur = c->fkr;  // FP32 copy of the current residual
  float* tmp = c->fkt;
  float* w = c->fkv;
  const bool sp = D == 3 && split0(c);  // the FP32 vectors in the colour-split layout
  if (sp)
    launch(c, kSlotVector, k_split_from, grid_for(n / 2), kThreads, cur, (const double*)r, (const double*)nullptr, L0.g,
           D);
  else
    launch(c, kSlotVector, k_convert<float, double>, nb, kThreads, cur, (const double*)r, n);
  double m = reduce_max_abs_f(c, cur, n, &st);
  if (st) return st;
  const dim3 blk(256, 1, 1);
  const dim3 grd(op3_blocks<D>(L0.g), 1, 1);
  auto step_along = [&](const float* d, int bit) -> int {
    const float* e0 = L0.feta;
    if (sp)
      launch3(c, kSlotVector, k_visc_op_split, split_grid(L0.g), split_block_dim(L0.g, 2), d, (const float*)nullptr, w,
              e0, L0.g, fbeta, 1);
    else if (staged_op(c, kSlotVector, d, nullptr, w, e0, L0.g, fbeta, 1))
      ;
    else if (any_per(c->g))
      launch3(c, kSlotVector, k_visc_op3<D, float, true, true>, grd, blk, d, (const float*)nullptr, w, e0, e0, e0, L0.g,
            fbeta, 1);
    else
      launch3(c, kSlotVector, k_visc_op3<D, float, true, false>, grd, blk, d, (const float*)nullptr, w, e0, e0, e0, L0.g,
            fbeta, 1);
    const double rw = reduce_dot_f(c, cur, w, n, &st);
    if (st) return st;
    const double ww = reduce_dot_f(c, w, w, n, &st);
    if (st) return st;
    if (!(ww > 0.0) || !std::isfinite(rw)) return HBF_OK;
    const double a = rw / ww;
    launch(c, kSlotVector, k_axmy<float>, nb, kThreads, tmp, (const float*)cur, (float)a, (const float*)w, n);
    const double m1 = reduce_max_abs_f(c, tmp, n, &st);
    if (st) return st;
    if (m1 < m) {
      if (sp) {
        launch(c, kSlotVector, k_split_add, grid_for(n / 2), kThreads, x, a, d, L0.g, D);
        launch(c, kSlotVector, k_split_add, grid_for(n / 2), kThreads, r, -a, (const float*)w, L0.g, D);
      } else {
        launch(c, kSlotVector, k_add_scaled_f32, nb, kThreads, x, a, d, n);
        launch(c, kSlotVector, k_add_scaled_f32, nb, kThreads, r, -a, (const float*)w, n);
      }
      float* t = cur;
      cur = tmp;
      tmp = t;
      m = m1;
      *used |= bit;
    }
    return HBF_OK;
  };
  if (c->vprev_ok && c->vprev32 && (st = step_along(c->vprev32, 1))) return st;
  if (c->vguess_mode >= 2 && c->vnet && m > 0.0 && visc_net_direction(c, cur, 1.0 / m, c->fke) &&
      (st = step_along(c->fke, 2)))
    return st;
  if ((st = cuda_check(c, cudaGetLastError(), "viscous guess"))) return st;
  *rn = reduce_max_abs(c, r, n, &st);
  return st;
}

template <int D>
static int solve_viscous_mixed(hbf_ctx* c, double beta, const double* b_in, double* x, hbf_solve_stats* out) {
  const SolverCfg& cfg = c->cfg;
  Level& L0 = c->lv[0];
  const long long n = (long long)D * L0.g.ncell;
  const size_t bytes = (size_t)n * sizeof(double);
  const size_t fbytes = (size_t)n * sizeof(float);
  const int nb = grid_for(n);
  double *kb = c->kb, *r = c->kr;
  float *fr = c->fkr, *frh = c->fkrh, *fp = c->fkp, *fv = c->fkv, *fs = c->fks, *ft = c->fkt, *fph = c->fkph,
        *fsh = c->fksh, *fe = c->fke;
  ViscProblem<D, double> P(c, x, beta, false);
  const float fbeta = (float)beta;
  const bool sp = D == 3 && split0(c);  // the FP32 level-0 vectors in the colour-split layout
  if (c->split_last != (int)sp) c->vprev_ok = false;  // the kept increment is in the other layout
  c->split_last = (int)sp;
  int st = 0;
  auto true_residual = [&]() -> double {
    cudaMemcpyAsync(L0.vb, kb, bytes, cudaMemcpyDeviceToDevice, c->stream);
    P.resid(0);
    cudaMemcpyAsync(r, L0.vr, bytes, cudaMemcpyDeviceToDevice, c->stream);
    return reduce_max_abs(c, r, n, &st);
  };
  // the V-cycle reads q as its level-0 right-hand side in place (the fused
  // tail starts on level 1 or below, so its argument records never hold level
  // 0's array)
  auto precond = [&](const float* q, float* z) {
    ViscProblem<D, float> Pz(c, z, beta, true);
    Pz.b0 = q;
    launch(c, kSlotTransfer, k_zero<float>, nb, kThreads, z, n);
    vcycle(Pz, 0, cfg);
  };
  const dim3 blk(256, 1, 1);
  const dim3 grd(op3_blocks<D>(L0.g), 1, 1);
  auto apply0 = [&](const float* q, float* o) {
    const float* e0 = L0.feta;
    if (sp) {
      launch3(c, kSlotViscResid, k_visc_op_split, split_grid(L0.g), split_block_dim(L0.g, 2), q, (const float*)nullptr, o,
              e0, L0.g, fbeta, 1);
      return;
    }
    if (staged_op(c, kSlotViscResid, q, nullptr, o, e0, L0.g, fbeta, 1)) return;
    if (any_per(c->g))
      launch3(c, kSlotViscResid, k_visc_op3<D, float, true, true>, grd, blk, q, (const float*)nullptr, o, e0, e0, e0, L0.g,
            fbeta, 1);
    else
      launch3(c, kSlotViscResid, k_visc_op3<D, float, true, false>, grd, blk, q, (const float*)nullptr, o, e0, e0, e0, L0.g,
            fbeta, 1);
  };
  if ((st = cuda_check(c, cudaMemcpyAsync(kb, b_in, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy rhs")))
    return st;
  double bnorm = reduce_max_abs(c, kb, n, &st);
  if (st) return st;
  double rn = true_residual();
  if (st) return st;
  double r0 = rn;
  if (bnorm == 0.0) bnorm = rn;
  const double tol = cfg.rtol * bnorm;
  int used = 0;
  if (c->vguess_mode > 0 && rn > tol && std::isfinite(rn) && (st = visc_guess<D>(c, beta, x, r, &rn, &used)))
    return st;
  if (c->vrecord && c->vres0) {
    cudaMemcpyAsync(c->vres0, r, bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->vcorr, x, bytes, cudaMemcpyDeviceToDevice, c->stream);  // the start; hbf_step subtracts
  }
  int it = 0;
  while (rn > tol && it < cfg.max_cycles && std::isfinite(rn)) {
    if (sp)
      launch(c, kSlotTransfer, k_split_from, grid_for(n / 2), kThreads, fr, (const double*)r, (const double*)nullptr,
             L0.g, D);
    else
      launch(c, kSlotTransfer, k_convert<float, double>, nb, kThreads, fr, (const double*)r, n);
    launch(c, kSlotTransfer, k_zero<float>, nb, kThreads, fe, n);
    cudaMemcpyAsync(frh, fr, fbytes, cudaMemcpyDeviceToDevice, c->stream);
    launch(c, kSlotTransfer, k_zero<float>, nb, kThreads, fv, n);
    launch(c, kSlotTransfer, k_zero<float>, nb, kThreads, fp, n);
    double in_norm = reduce_max_abs_f(c, fr, n, &st);
    if (st) return st;
    const double in_tol = c->inner_drop * in_norm;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    // the fused vector kernels need 16-byte aligned vectors (cudaMalloc'd)
    const bool fused = aligned16(fr) && aligned16(fs) && aligned16(ft) && aligned16(frh);
    double rho_next = 0.0;  // r^.r of the updated r, from the fused update
    for (int k = 0; k < kInnerMax && it < cfg.max_cycles; ++k) {
      double rho1 = (fused && k > 0) ? rho_next : reduce_dot_f(c, frh, fr, n, &st);
      if (st) return st;
      if (rho1 == 0.0 || !std::isfinite(rho1)) break;
      double bt = (rho1 / rho) * (alpha / omega);
      launch(c, kSlotVector, k_bicg_p<float>, nb, kThreads, fp, (const float*)fr, (const float*)fv, (float)bt,
             (float)omega, n);
      precond(fp, fph);
      apply0(fph, fv);
      double den = reduce_dot_f(c, frh, fv, n, &st);
      if (st) return st;
      if (den == 0.0 || !std::isfinite(den)) break;
      alpha = rho1 / den;
      launch(c, kSlotVector, k_axmy<float>, nb, kThreads, fs, (const float*)fr, (float)alpha, (const float*)fv, n);
      precond(fs, fsh);
      apply0(fsh, ft);
      double tt, ts;
      if (fused) {
        if ((st = reduce_dot2_f(c, ft, fs, n, &tt, &ts))) return st;
      } else {
        tt = reduce_dot_f(c, ft, ft, n, &st);
        if (st) return st;
        ts = reduce_dot_f(c, ft, fs, n, &st);
        if (st) return st;
      }
      omega = tt > 0.0 ? ts / tt : 0.0;
      launch(c, kSlotVector, k_bicg_x<float>, nb, kThreads, fe, (const float*)fph, (const float*)fsh, (float)alpha,
             (float)omega, n);
      double rr;
      if (fused) {
        // r = s - omega t with max |r| and r^.r of the new r in one pass
        launch(c, kSlotVector, k_axmy_red_f4, kRedBlocks, kThreads, fr, (const float*)fs, (float)omega,
               (const float*)ft, (const float*)frh, n, c->partial);
        if ((st = read_results2(c, &rr, &rho_next))) return st;
      } else {
        launch(c, kSlotVector, k_axmy<float>, nb, kThreads, fr, (const float*)fs, (float)omega, (const float*)ft, n);
        rr = reduce_max_abs_f(c, fr, n, &st);
        if (st) return st;
      }
      rho = rho1;
      ++it;
      if (rr <= in_tol || omega == 0.0 || !std::isfinite(rr)) break;
    }
    if (sp)
      launch(c, kSlotTransfer, k_split_add, grid_for(n / 2), kThreads, x, 1.0, (const float*)fe, L0.g, D);
    else
      launch(c, kSlotTransfer, k_add_f32, nb, kThreads, x, (const float*)fe, n);
    rn = true_residual();
    if (st) return st;
  }
  if ((st = cuda_check(c, cudaGetLastError(), "viscous solve"))) return st;
  st = finish(c, it, r0, rn, bnorm, tol, out);
  if (out) out->guess = used;
  return st;
}

template <int D>
static int solve_viscous_d(hbf_ctx* c, double beta, const double* b_in, double* x, hbf_solve_stats* out) {
  build_eta_levels<D>(c);
  c->dense[0].valid = false;  // new viscosity and dt: rebuild the bottom inverse
  if (c->precision == HBF_MIXED) return solve_viscous_mixed<D>(c, beta, b_in, x, out);
  const SolverCfg& cfg = c->cfg;
  Level& L0 = c->lv[0];
  const long long n = (long long)D * L0.g.ncell;
  const size_t bytes = (size_t)n * sizeof(double);
  const int nb = grid_for(n);
  double *kb = c->kb, *r = c->kr, *rh = c->krh, *p = c->kp, *v = c->kv, *s = c->ks, *t = c->kt, *ph = c->kph,
         *sh = c->ksh;
  ViscProblem<D, double> P(c, x, beta, false);
  ViscProblem<D, float> Pre32(c, L0.fvx, beta, true);
  const bool mixed = c->precision == HBF_MIXED;
  int st;
  auto true_residual = [&]() -> double {
    cudaMemcpyAsync(L0.vb, kb, bytes, cudaMemcpyDeviceToDevice, c->stream);
    P.resid(0);
    cudaMemcpyAsync(r, L0.vr, bytes, cudaMemcpyDeviceToDevice, c->stream);
    return reduce_max_abs(c, r, n, &st);
  };
  // z = M^{-1} q
  auto precond = [&](const double* q, double* z) {
    if (mixed) {
      launch(c, kSlotTransfer, k_convert<float, double>, nb, kThreads, L0.fvb, q, n);
      launch(c, kSlotTransfer, k_zero<float>, nb, kThreads, L0.fvx, n);
      vcycle(Pre32, 0, cfg);
      launch(c, kSlotTransfer, k_convert<double, float>, nb, kThreads, z, (const float*)L0.fvx, n);
    } else {
      ViscProblem<D, double> Pz(c, z, beta, true);
      Pz.b0 = q;  // read in place, as in the mixed solve
      launch(c, kSlotTransfer, k_zero<double>, nb, kThreads, z, n);
      vcycle(Pz, 0, cfg);
    }
  };
  auto apply0 = [&](const double* q, double* out_) {
    const dim3 blk(256, 1, 1);
    const dim3 grd(op3_blocks<D>(L0.g), 1, 1);
    if (any_per(c->g))
      launch3(c, l0slot(), k_visc_op3<D, double, false, true>, grd, blk, q, (const double*)nullptr, out_, (const double*)L0.ef[0],
            (const double*)L0.ef[1], (const double*)L0.ef[2], L0.g, beta, 1);
    else
      launch3(c, l0slot(), k_visc_op3<D, double, false, false>, grd, blk, q, (const double*)nullptr, out_, (const double*)L0.ef[0],
            (const double*)L0.ef[1], (const double*)L0.ef[2], L0.g, beta, 1);
  };
  if ((st = cuda_check(c, cudaMemcpyAsync(kb, b_in, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy rhs")))
    return st;
  double bnorm = reduce_max_abs(c, kb, n, &st);
  if (st) return st;
  double rn = true_residual();
  if (st) return st;
  double r0 = rn;
  if (bnorm == 0.0) bnorm = rn;
  const double tol = cfg.rtol * bnorm;
  int it = 0;
  while (rn > tol && it < cfg.max_cycles && std::isfinite(rn)) {
    cudaMemcpyAsync(rh, r, bytes, cudaMemcpyDeviceToDevice, c->stream);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    launch(c, kSlotTransfer, k_zero<double>, nb, kThreads, v, n);
    launch(c, kSlotTransfer, k_zero<double>, nb, kThreads, p, n);
    while (it < cfg.max_cycles) {
      double rho1 = reduce_dot(c, rh, r, n, &st);
      if (st) return st;
      if (rho1 == 0.0 || !std::isfinite(rho1)) break;
      double bt = (rho1 / rho) * (alpha / omega);
      launch(c, kSlotVector, k_bicg_p<double>, nb, kThreads, p, (const double*)r, (const double*)v, bt, omega, n);
      precond(p, ph);
      apply0(ph, v);
      double den = reduce_dot(c, rh, v, n, &st);
      if (st) return st;
      if (den == 0.0 || !std::isfinite(den)) break;
      alpha = rho1 / den;
      launch(c, kSlotVector, k_axmy<double>, nb, kThreads, s, (const double*)r, alpha, (const double*)v, n);
      precond(s, sh);
      apply0(sh, t);
      double tt = reduce_dot(c, t, t, n, &st);
      if (st) return st;
      double ts = reduce_dot(c, t, s, n, &st);
      if (st) return st;
      omega = tt > 0.0 ? ts / tt : 0.0;
      launch(c, kSlotVector, k_bicg_x<double>, nb, kThreads, x, (const double*)ph, (const double*)sh, alpha, omega, n);
      launch(c, kSlotVector, k_axmy<double>, nb, kThreads, r, (const double*)s, omega, (const double*)t, n);
      rho = rho1;
      ++it;
      double rr = reduce_max_abs(c, r, n, &st);
      if (st) return st;
      if (rr <= tol || omega == 0.0 || !std::isfinite(rr)) break;
    }
    rn = true_residual();
    if (st) return st;
  }
  if ((st = cuda_check(c, cudaGetLastError(), "viscous solve"))) return st;
  return finish(c, it, r0, rn, bnorm, tol, out);
}

int solve_viscous(hbf_ctx* c, double beta, const double* rhs, double* u, hbf_solve_stats* s) {
  int st = launch_eta_faces(c);
  if (st) return st;
  st = c->dim == 2 ? solve_viscous_d<2>(c, beta, rhs, u, s) : solve_viscous_d<3>(c, beta, rhs, u, s);
  const int se = take_sweep_err(c);
  return st ? st : se;
}

template <int D>
static int solve_mac_d(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  MacProblem<D, double> P(c, phi);
  if (c->precision == HBF_MIXED) {
    MacProblem<D, float> P32(c, c->lv[0].fcx);
    return mg_solve(P, &P32, rhs, s);
  }
  return mg_solve(P, nullptr, rhs, s);
}

int solve_mac(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  return c->dim == 2 ? solve_mac_d<2>(c, rhs, phi, s) : solve_mac_d<3>(c, rhs, phi, s);
}

template <int D>
static int solve_nodal_d(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  NodalProblem<D, double> P(c, phi);
  if (c->precision == HBF_MIXED) {
    NodalProblem<D, float> P32(c, c->lv[0].fnx);
    return mg_solve(P, &P32, rhs, s);
  }
  return mg_solve(P, nullptr, rhs, s);
}

int solve_nodal(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s) {
  return c->dim == 2 ? solve_nodal_d<2>(c, rhs, phi, s) : solve_nodal_d<3>(c, rhs, phi, s);
}

int nodal_residual(hbf_ctx* c, const double* b, const double* x, double* r) {
  if (c->dim == 2) {
    if (any_per(c->g))
      launch(c, kSlotNodalResid, k_nodal_resid<2, double, true>, grid_for(c->g.nnode), kThreads, x, b, r, c->g);
    else
      launch(c, kSlotNodalResid, k_nodal_resid<2, double, false>, grid_for(c->g.nnode), kThreads, x, b, r, c->g);
  } else {
    if (any_per(c->g))
      launch(c, kSlotNodalResid, k_nodal_resid<3, double, true>, grid_for(c->g.nnode), kThreads, x, b, r, c->g);
    else
      launch(c, kSlotNodalResid, k_nodal_resid<3, double, false>, grid_for(c->g.nnode), kThreads, x, b, r, c->g);
  }
  return cuda_check(c, cudaGetLastError(), "nodal residual");
}

void nodal_restrict(hbf_ctx* c, int l, const double* fine, double* coarse) {
  const Level &F = c->lv[l], &C = c->lv[l + 1];
  if (c->dim == 2) {
    if (any_per(c->g))
      launch(c, kSlotTransfer, k_restrict_nodes<2, double, true>, grid_for(C.g.nnode), kThreads, fine, coarse, F.g, C.g);
    else
      launch(c, kSlotTransfer, k_restrict_nodes<2, double, false>, grid_for(C.g.nnode), kThreads, fine, coarse, F.g, C.g);
  } else {
    if (any_per(c->g))
      launch(c, kSlotTransfer, k_restrict_nodes<3, double, true>, grid_for(C.g.nnode), kThreads, fine, coarse, F.g, C.g);
    else
      launch(c, kSlotTransfer, k_restrict_nodes<3, double, false>, grid_for(C.g.nnode), kThreads, fine, coarse, F.g, C.g);
  }
}

void nodal_prolong_add(hbf_ctx* c, int l, double* fine, const double* coarse) {
  const Level &F = c->lv[l], &C = c->lv[l + 1];
  if (c->dim == 2)
    launch(c, kSlotTransfer, k_prolong_nodes_add<2, double>, grid_for(F.g.nnode), kThreads, fine, coarse, F.g, C.g);
  else
    launch(c, kSlotTransfer, k_prolong_nodes_add<3, double>, grid_for(F.g.nnode), kThreads, fine, coarse, F.g, C.g);
}

void cell_restrict_f(hbf_ctx* c, int l, const float* fine, float* coarse) {
  const Level &F = c->lv[l], &C = c->lv[l + 1];
  const long long n = (long long)c->dim * C.g.ncell;
  if (c->dim == 2)
    launch(c, kSlotTransfer, k_restrict_cells<2, float>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 2);
  else if (l == 0 && split0(c))  // the FP32 level-0 vectors of the mixed viscous solve
    launch(c, kSlotTransfer, k_restrict_cells<3, float, true>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 3);
  else
    launch(c, kSlotTransfer, k_restrict_cells<3, float>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 3);
}

void cell_restrict_d(hbf_ctx* c, int l, const double* fine, double* coarse, int ncomp) {
  const Level &F = c->lv[l], &C = c->lv[l + 1];
  const long long n = (long long)ncomp * C.g.ncell;
  if (c->dim == 2)
    launch(c, kSlotTransfer, k_restrict_cells<2, double>, grid_for(n), kThreads, fine, coarse, F.g, C.g, ncomp);
  else
    launch(c, kSlotTransfer, k_restrict_cells<3, double>, grid_for(n), kThreads, fine, coarse, F.g, C.g, ncomp);
}

void cell_prolong_add_f(hbf_ctx* c, int l, float* fine, const float* coarse) {
  const Level &F = c->lv[l], &C = c->lv[l + 1];
  const long long n = (long long)c->dim * C.g.ncell;
  // odd reflection at the walls: a correction of the Dirichlet problem
  if (c->dim == 2) {
    if (any_per(c->g))
      launch(c, kSlotTransfer, k_prolong_cells_add_c<2, float, true>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 2, -1.f);
    else
      launch(c, kSlotTransfer, k_prolong_cells_add_c<2, float, false>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 2, -1.f);
  } else if (l == 0 && split0(c)) {  // the FP32 level-0 vectors of the mixed viscous solve
    launch(c, kSlotTransfer, k_prolong_cells_add_c<3, float, false, true>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 3,
           -1.f);
  } else {
    if (any_per(c->g))
      launch(c, kSlotTransfer, k_prolong_cells_add_c<3, float, true>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 3, -1.f);
    else
      launch(c, kSlotTransfer, k_prolong_cells_add_c<3, float, false>, grid_for(n), kThreads, fine, coarse, F.g, C.g, 3, -1.f);
  }
}

int visc_after_solve(hbf_ctx* c, const double* ustar, const double* u) {
  const long long n = (long long)c->dim * c->g.ncell;
  if (c->vguess_mode > 0 && c->vprev32) {
    if (c->dim == 3 && split0(c))  // kept in the layout of the FP32 vectors of the next solve
      launch(c, kSlotVector, k_split_from, grid_for(n / 2), kThreads, c->vprev32, ustar, u, c->lv[0].g, 3);
    else
      launch(c, kSlotVector, k_diff_to_f32, grid_for(n), kThreads, c->vprev32, ustar, u, n);
    c->vprev_ok = true;
  }
  if (c->vrecord && c->vcorr) launch(c, kSlotVector, k_rsub, grid_for(n), kThreads, ustar, c->vcorr, n);  // u* - start
  return cuda_check(c, cudaGetLastError(), "viscous increment");
}

void axmy(hbf_ctx* c, double* out, const double* x, double a, const double* y, long long n) {
  launch(c, kSlotVector, k_axmy<double>, grid_for(n), kThreads, out, x, a, y, n);
}

int tensor_lu(hbf_ctx* c, const double* u, double* out) {
  const Level& L = c->lv[0];
  if (c->dim == 2)
    launch(c, kSlotExplicit, k_tensor_lu<2, double>, grid_for(xi_count<2>(L.g), 152 * 24), kThreads, u, out,
           (const double*)L.ef[0], (const double*)L.ef[1], (const double*)L.ef[2], L.g, 0);
  else
    launch(c, kSlotExplicit, k_tensor_lu<3, double>, grid_for(xi_count<3>(L.g), 152 * 24), kThreads, u, out,
           (const double*)L.ef[0], (const double*)L.ef[1], (const double*)L.ef[2], L.g, 0);
  return cuda_check(c, cudaGetLastError(), "k_tensor_lu");
}

// exact bottom solve of problem `kind` (0 viscous, 1 MAC, 2 nodal) for a
// context whose coarsest level is small enough; returns false otherwise
bool ensure_dense(hbf_ctx* c, int kind, double beta) {
  const int l = (int)c->lv.size() - 1;
  const Level& L = c->lv[l];
  const long long n = kind == 0 ? (long long)c->dim * L.g.ncell : (kind == 1 ? L.g.ncell : L.g.nnode);
  if (n > kDenseMax) return false;
  if (!c->dense[kind].valid) {
    if (c->dim == 2)
      build_dense<2>(c, kind, l, n, beta);
    else
      build_dense<3>(c, kind, l, n, beta);
  }
  return true;
}

}  // namespace hb

extern "C" int hbf_cfl_dt_noalloc(const double* u_dev, int64_t n, double h, double cfl, double* dt_dev,
                                  void* stream) {
  using namespace hb;
  if (!u_dev || !dt_dev || n < 1 || !(h > 0.0) || !(cfl > 0.0)) return HBF_ERR_ARG;
  if (n > kNoAllocMaxN) return HBF_ERR_ARG;  // more elements than the static partial array covers
  int st = 0;
  double* part = noalloc_scratch(&st);
  if (st) return st;
  // an error left pending by earlier work of the caller is not this call's:
  // leave it for the caller to read and launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return HBF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int nb = (int)((n + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
  k_noalloc_maxabs_partial<<<nb, kThreads, 0, s>>>(u_dev, (long long)n, part);
  k_noalloc_cfl_final<<<1, 1024, 0, s>>>(part, nb, h, cfl, dt_dev);
  return cudaGetLastError() == cudaSuccess ? HBF_OK : HBF_ERR_CUDA;
}
