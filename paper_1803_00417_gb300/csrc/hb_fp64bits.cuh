// FP64 sign tests, magnitude comparisons and scalings by 2 and 1/2 on the
// integer pipe.  GB300 issues FP64 instructions at 1/64 of its FP32 rate
// (2 per SM and cycle), and the limiter and upwind choices of the predictor
// are comparisons and exact scalings: on the two 32-bit halves of the bit
// pattern they cost a few integer instructions each and give the IEEE answer
// for every non-NaN operand (+0 and -0 both count as zero; x/2 and 2x
// rounded to nearest even, subnormals and overflow included).  The halves are
// taken with the hi/lo intrinsics so that no 64-bit pattern is left for the
// compiler to turn back into an FP64 compare or fabs.
#pragma once
#include <cstring>

namespace hb {

struct DHalves {
  int hi;       // sign, 11 exponent bits, top 20 significand bits
  unsigned lo;  // low 32 significand bits
};

__host__ __device__ __forceinline__ DHalves dsplit(double x) {
#ifdef __CUDA_ARCH__
  return DHalves{__double2hiint(x), (unsigned)__double2loint(x)};
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  return DHalves{(int)(unsigned)(b >> 32), (unsigned)b};
#endif
}

__host__ __device__ __forceinline__ double djoin(int hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double(hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | lo;
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

constexpr int kDMag = 0x7fffffff;
constexpr int kDSign = (int)0x80000000u;

// x == 0, x > 0, x < 0
__host__ __device__ __forceinline__ bool dzero(double x) {
  const DHalves d = dsplit(x);
  return ((unsigned)(d.hi & kDMag) | d.lo) == 0u;
}
__host__ __device__ __forceinline__ bool dpos(double x) {
  const DHalves d = dsplit(x);
  return d.hi >= 0 && ((unsigned)d.hi | d.lo) != 0u;
}
__host__ __device__ __forceinline__ bool dneg(double x) {
  const DHalves d = dsplit(x);
  return d.hi < 0 && ((unsigned)(d.hi & kDMag) | d.lo) != 0u;
}

// a and b nonzero with the same sign (a b > 0 unless the product underflows)
__host__ __device__ __forceinline__ bool dsame_sign(double a, double b) {
  const DHalves x = dsplit(a), y = dsplit(b);
  return ((unsigned)(x.hi & kDMag) | x.lo) != 0u && ((unsigned)(y.hi & kDMag) | y.lo) != 0u && (x.hi ^ y.hi) >= 0;
}

// min(|a|, |b|): the smaller magnitude pattern (finite operands order like
// their patterns)
__host__ __device__ __forceinline__ double dminabs(double a, double b) {
  const DHalves x = dsplit(a), y = dsplit(b);
  const int xh = x.hi & kDMag, yh = y.hi & kDMag;
  const bool xl = xh < yh || (xh == yh && x.lo < y.lo);
  return xl ? djoin(xh, x.lo) : djoin(yh, y.lo);
}

// sign(v) min(|v|, lim) with sign(0) = 0, for lim >= +0
__host__ __device__ __forceinline__ double dsgn_min(double v, double lim) {
  if (dzero(v)) return 0.0;
  const DHalves m = dsplit(dminabs(v, lim));
  return djoin(m.hi | (dsplit(v).hi & kDSign), m.lo);
}

// x / 2: one off the exponent, or (subnormal results) the significand
// shifted right by one with ties to even
__host__ __device__ __forceinline__ double dhalf(double x) {
  const DHalves d = dsplit(x);
  const int e = (d.hi >> 20) & 0x7ff;
  if (e >= 2 && e < 0x7ff) return djoin(d.hi - 0x100000, d.lo);
  if (e == 0x7ff) return x;
  const unsigned mhi = (unsigned)(d.hi & 0x000fffff) | (e == 1 ? 0x00100000u : 0u);
  unsigned rhi = mhi >> 1, rlo = (d.lo >> 1) | (mhi << 31);
  if ((d.lo & 1u) && (rlo & 1u)) {
    rlo += 1u;
    rhi += (rlo == 0u);
  }
  return djoin((int)(rhi | (unsigned)(d.hi & kDSign)), rlo);
}

// 2 x: one onto the exponent, subnormals shifted left (exact), +-inf past
// the largest finite exponent
__host__ __device__ __forceinline__ double dtwice(double x) {
  const DHalves d = dsplit(x);
  const int e = (d.hi >> 20) & 0x7ff;
  if (e >= 1 && e <= 0x7fd) return djoin(d.hi + 0x100000, d.lo);
  if (e == 0x7ff) return x;
  if (e == 0x7fe) return djoin((d.hi & kDSign) | 0x7ff00000, 0u);
  const unsigned mhi = (unsigned)(d.hi & 0x000fffff);
  return djoin((int)(((mhi << 1) | (d.lo >> 31)) | (unsigned)(d.hi & kDSign)), d.lo << 1);
}

}  // namespace hb
