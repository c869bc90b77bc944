// FP64 elementary functions used by the Cayley-Hamilton coefficients.
//
// GB300 issues FP64 instructions at 1/64 of the FP32 rate, so each function
// here is built to take few FP64 instructions: a hardware approximation
// (MUFU or an FP32 library call) as the seed, refined by Newton iterations in
// FP64, or a truncated Taylor series in FP64.  Every result is accurate to a
// few FP64 ulps on the ranges where it is used; the stout parity tests
// against the FP64 oracle (1e-12 per link element) exercise all of them.
#pragma once

#include <cuda_runtime.h>

namespace lq {

// float -> double and double -> float through the IEEE-754 bit fields on the
// integer pipe (the hardware conversions issue on the FP64 pipe, which is the
// bottleneck).  f2d: exact for normal numbers and zero (FP32 subnormals become
// signed zero, inf/NaN keep their class).  d2f: round to nearest, ties to
// even, for results in the FP32 normal range; below it signed zero (FP32
// subnormals flushed), above it infinity, NaN kept.  No branch and no
// hardware conversion: a fallback to the hardware conversion, even one that
// no lane takes, is issued to the FP64 pipe by the whole warp.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned ed = e == 0u ? 0u : (e == 255u ? 2047u : e + 896u);
  const unsigned hi = (u & 0x80000000u) | (ed << 20) | (e == 0u ? 0u : ((u & 0x7fffffu) >> 3));
  const unsigned lo = e == 0u ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u, mag = hi & 0x7fffffffu;
  const int e = (int)(mag >> 20) - 896;
  unsigned f = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  f += (rest > 0x10000000u ? 1u : 0u) | (rest == 0x10000000u ? (f & 1u) : 0u);   // a carry may reach inf
  const bool nan = mag > 0x7ff00000u || (mag == 0x7ff00000u && lo != 0u);
  f = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u | (nan ? 0x00400000u : 0u)) : f);
  return __uint_as_float(f);
}

// NR = number of Newton steps after the FP32 seed (relative error ~2^-22):
// 2 reaches FP64 rounding (used by the FP64 path), 1 gives ~1e-13, far below
// the FP32 rounding of the FP32 path's matrix algebra.

// 1/sqrt(a), a > 0 and a normal FP32 number: FP32 seed, Newton steps
// r <- r (3/2 - a r^2 / 2).
template <int NR = 2> __device__ __forceinline__ double rsqrt_nr(double a) {
  double r = f2d(rsqrtf(d2f(a)));
  const double ha = 0.5 * a;
#pragma unroll
  for (int i = 0; i < NR; ++i) r = r * fma(-ha * r, r, 1.5);
  return r;
}

// 1/a, a a normal FP32 number: FP32 seed, Newton steps r <- r + r (1 - a r).
template <int NR = 2> __device__ __forceinline__ double rcp_nr(double a) {
  double r = f2d(__frcp_rn(d2f(a)));
#pragma unroll
  for (int i = 0; i < NR; ++i) r = fma(r, fma(-a, r, 1.0), r);
  return r;
}

// y = cos(arccos(x)/3) for x in [0, 1]: the root in [cos(pi/6), 1] of the
// Chebyshev cubic 4y^3 - 3y = x (cos 3t = 4cos^3 t - 3cos t), refined by two
// Newton steps from an FP32 evaluation.  f'(y) = 12y^2 - 3 >= 6 on that range,
// so an FP32 reciprocal of f' suffices for the step.
template <int NR = 2> __device__ __forceinline__ double cos_third_acos(double x) {
  double y = f2d(cosf(acosf(d2f(x)) * (1.0f / 3.0f)));
#pragma unroll
  for (int it = 0; it < NR; ++it) {
    const double y2 = y * y;
    const double f = fma(y, fma(4.0, y2, -3.0), -x);
    const double fp = fma(12.0, y2, -3.0);
    y = fma(-f, f2d(__frcp_rn(d2f(fp))), y);
  }
  return y;
}

// sin and cos of |r| <= pi/4 (a little beyond is fine) from their Taylor
// series, truncated after r^15 and r^16 (next terms < 6e-17 relative).
__device__ __forceinline__ void sincos_taylor(double r, double* s, double* c) {
  const double r2 = r * r;
  double ps = -1.0 / 1307674368000.0;  // -1/15!
  ps = fma(ps, r2, 1.0 / 6227020800.0);  // 1/13!
  ps = fma(ps, r2, -1.0 / 39916800.0);   // -1/11!
  ps = fma(ps, r2, 1.0 / 362880.0);      // 1/9!
  ps = fma(ps, r2, -1.0 / 5040.0);       // -1/7!
  ps = fma(ps, r2, 1.0 / 120.0);         // 1/5!
  ps = fma(ps, r2, -1.0 / 6.0);          // -1/3!
  *s = fma(r * r2, ps, r);
  double pc = 1.0 / 20922789888000.0;    // 1/16!
  pc = fma(pc, r2, -1.0 / 87178291200.0);  // -1/14!
  pc = fma(pc, r2, 1.0 / 479001600.0);     // 1/12!
  pc = fma(pc, r2, -1.0 / 3628800.0);      // -1/10!
  pc = fma(pc, r2, 1.0 / 40320.0);         // 1/8!
  pc = fma(pc, r2, -1.0 / 720.0);          // -1/6!
  pc = fma(pc, r2, 1.0 / 24.0);            // 1/4!
  pc = fma(pc, r2, -0.5);                  // -1/2!
  *c = fma(r2, pc, 1.0);
}

// cos(w) and sin(w)/w from w^2 alone, for w^2 <= (pi/4)^2 (same series).
__device__ __forceinline__ void cos_sinc_from_sq(double w2, double* cw, double* xi0) {
  double ps = -1.0 / 1307674368000.0;
  ps = fma(ps, w2, 1.0 / 6227020800.0);
  ps = fma(ps, w2, -1.0 / 39916800.0);
  ps = fma(ps, w2, 1.0 / 362880.0);
  ps = fma(ps, w2, -1.0 / 5040.0);
  ps = fma(ps, w2, 1.0 / 120.0);
  ps = fma(ps, w2, -1.0 / 6.0);
  *xi0 = fma(w2, ps, 1.0);
  double pc = 1.0 / 20922789888000.0;
  pc = fma(pc, w2, -1.0 / 87178291200.0);
  pc = fma(pc, w2, 1.0 / 479001600.0);
  pc = fma(pc, w2, -1.0 / 3628800.0);
  pc = fma(pc, w2, 1.0 / 40320.0);
  pc = fma(pc, w2, -1.0 / 720.0);
  pc = fma(pc, w2, 1.0 / 24.0);
  pc = fma(pc, w2, -0.5);
  *cw = fma(w2, pc, 1.0);
}

// xi1(w) = cos(w)/w^2 - sin(w)/w^3 = xi0'(w)/w from w^2, for w^2 <= (pi/4)^2:
// sum_j (-1)^(j+1) (2j+2) w^(2j) / (2j+3)!, truncated after j = 7 (next term
// < 1e-15 relative).
__device__ __forceinline__ double xi1_from_sq(double w2) {
  double p = 16.0 / 355687428096000.0;    // +16/17!
  p = fma(p, w2, -14.0 / 1307674368000.0);  // -14/15!
  p = fma(p, w2, 12.0 / 6227020800.0);      // +12/13!
  p = fma(p, w2, -10.0 / 39916800.0);       // -10/11!
  p = fma(p, w2, 8.0 / 362880.0);           // +8/9!
  p = fma(p, w2, -6.0 / 5040.0);            // -6/7!
  p = fma(p, w2, 4.0 / 120.0);              // +4/5!
  return fma(p, w2, -2.0 / 6.0);            // -2/3!
}

// sin and cos of any finite x: reduction x = k pi/2 + r with pi/2 split in two
// doubles (Cody & Waite, "Software Manual for the Elementary Functions",
// 1980) and a fused multiply-add per part, then the quadrant of k.  Used for
// |x| < 2^20; larger arguments (never produced by a stout step with a sane
// rho) go to the CUDA library.
__device__ __forceinline__ void sincos_red(double x, double* s, double* c) {
  if (fabs(x) <= 0.78539816339744831) {
    sincos_taylor(x, s, c);
    return;
  }
  if (!(fabs(x) < 1048576.0)) {
    sincos(x, s, c);
    return;
  }
  // (a rho that produces |x| >= 2^20 has no physical use; the library covers it)
  const double k = rint(x * 0.63661977236758134);  // 2/pi
  double r = fma(-k, 1.5707963267948966, x);       // pi/2, leading double
  r = fma(-k, 6.123233995736766e-17, r);            // pi/2 - leading double
  double sr, cr;
  sincos_taylor(r, &sr, &cr);
  const int q = ((int)k) & 3;
  *s = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
  *c = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
}

}  // namespace lq
