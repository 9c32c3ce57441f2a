// Float32 mean of an exact double-float sum, without binary64 arithmetic.
//
// A voxel's mean and covariance (Sec. III-A: the voxel Gaussian averages the
// points' means and covariances) are defined as the binary64 sum divided by N
// in binary64, rounded to float32: f = RN32(RN64(RN64(S) / N)).  The build
// sums exactly in float32 pairs (S = hi + lo, hi = RN(hi + lo)), so only the
// division remains.  On a GPU whose binary64 rate is a small fraction of its
// float32 rate, it is done here in float32:
//
//   q  = candidate float32 quotient of |S| / N (|S| RN(1/N), then one Newton
//        correction);
//   M+, M- = the midpoints between q and its float32 neighbours;
//   z+- = |S| - M+- N, evaluated exactly: q N = p + e (FMA split), |hi| - p is
//        exact (Sterbenz), d - e -+ N u / 2 is a float sum checked to be exact
//        (TwoSum error 0), and RN(W + lo) has exactly the sign of W + lo;
//   q steps until M- <= x <= M+ for the quotient x = |S| / N.
//
// Then RN32(x) = q, or the even neighbour when x is a midpoint (z = 0; then
// S = M N has at most 49 significant bits, so the binary64 evaluation is exact
// and rounds the tie to even as well).  Double rounding through binary64 can
// change the result only when x lies within about 2^-52 |x| of a midpoint
// without being on it; such a quotient (|z| < 2^-50 |S|), a sum that is not
// exact as a float, or a magnitude outside the guarded range is reported as not
// certified, and the caller evaluates the binary64 definition instead.
//
// Host and device compile the same code: every operation is an explicitly
// rounded float32 operation (no contraction), so the host build of this
// header is a faithful model of the device code for tests.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define VGICP_HD __host__ __device__ __forceinline__
#else
#define VGICP_HD inline
#include <math.h>
#endif

namespace vgicp {
namespace mean32 {

VGICP_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
VGICP_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float r = a - b;
  return r;
#endif
}
VGICP_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
VGICP_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return ::fmaf(a, b, c);
#endif
}
VGICP_HD uint32_t bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
VGICP_HD float from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
VGICP_HD float fabs_(float f) { return from_bits(bits(f) & 0x7FFFFFFFu); }
// TwoSum (Knuth; Moeller): s = RN(a + b), e = a + b - s exactly.
VGICP_HD void two_sum_f(float a, float b, float& s, float& e) {
  s = add(a, b);
  const float bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
}

}  // namespace mean32

// Returns RN32(RN64(RN64(hi + lo) / n)) and sets ok, or clears ok (the caller
// then evaluates that definition in binary64).  Requires hi = RN32(hi + lo)
// (|lo| <= ulp(hi) / 2), as the exact double-float sums provide, and
// rN = RN32(1 / n) (shared by the components of one voxel).  Certified range:
// n <= 2^24 and 2^-60 <= |hi| <= 2^100, or hi = lo = 0.
VGICP_HD float mean_rn32(float hi, float lo, uint32_t n, float rN, bool& ok) {
  using namespace mean32;
  ok = false;
  if (hi == 0.0f) {
    ok = lo == 0.0f;
    return 0.0f;
  }
  if (n == 0u || n > (1u << 24)) return 0.0f;
  const float a = fabs_(hi);
  if (!(a >= 0x1p-60f && a <= 0x1p100f)) return 0.0f;  // also NaN and infinity
  const float l = hi < 0.0f ? -lo : lo;                 // |S| = a + l
  const float N = (float)n;                             // exact
  const float win = mul(a, 0x1p-50f);                   // double-rounding window
  float q = mul(a, rN);  // within 2 ulp of |S| / N
  {  // one Newton step: q + (|S| - q N) / N, then within about 1 ulp
    const float p = mul(q, N);
    const float R = add(sub(sub(a, p), fma(q, N, -p)), l);
    q = add(q, mul(R, rN));
  }
  for (int it = 0; it < 6; ++it) {
    const uint32_t qb = bits(q);
    const float p = mul(q, N);
    const float e = fma(q, N, -p);  // q N - p, exact
    const float d = sub(a, p);      // exact: p is within a factor 2 of a
    const float u = from_bits((qb & 0x7F800000u) - (23u << 23));  // spacing above q
    const float udn = (qb & 0x007FFFFFu) ? u : mul(u, 0.5f);       // spacing below q
    const float hu = mul(mul(u, N), 0.5f);                          // exact
    const float hd = mul(mul(udn, N), 0.5f);                        // exact
    float t, err;
    two_sum_f(d, -e, t, err);
    if (err != 0.0f) return 0.0f;
    float wu, wd, eu, ed;
    two_sum_f(t, -hu, wu, eu);
    two_sum_f(t, hd, wd, ed);
    if (eu != 0.0f || ed != 0.0f) return 0.0f;
    const float zu = add(wu, l);  // sign of |S| - M+ N
    const float zd = add(wd, l);  // sign of |S| - M- N
    if (zu > 0.0f) {
      q = from_bits(qb + 1u);
      continue;
    }
    if (zd < 0.0f) {
      q = from_bits(qb - 1u);
      continue;
    }
    float r = q;
    if (zu == 0.0f) {
      r = (qb & 1u) ? from_bits(qb + 1u) : q;  // tie at M+: the even one
    } else if (zd == 0.0f) {
      r = (qb & 1u) ? from_bits(qb - 1u) : q;  // tie at M-: the even one
    } else if (fabs_(zu) < win || fabs_(zd) < win) {
      return 0.0f;  // within the double-rounding window of a midpoint
    }
    ok = true;
    return hi < 0.0f ? -r : r;
  }
  return 0.0f;
}

}  // namespace vgicp

#undef VGICP_HD
