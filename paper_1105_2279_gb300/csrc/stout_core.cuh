// Per-link stout smearing arithmetic (Morningstar & Peardon 2004, Secs. II-III):
// staple sum, Omega = C U^dag, Q, Cayley-Hamilton coefficients f0,f1,f2 (always
// FP64), exp(iQ) = f0 + f1 Q + f2 Q^2, U' = exp(iQ) U, optional FP64 SU(3)
// re-projection.  Shared by the single-lattice, batched and backward kernels.
#pragma once

#include "fp64_math.cuh"
#include "lq_internal.h"
#include "su3.cuh"

namespace lq {

template <typename R>
__device__ __forceinline__ M3<R> ld_link(const typename vec2<R>::type* __restrict__ U, long long V,
                                         int dir, int s) {
  return ld_m3<R>(U + (long long)dir * 9 * V + s, V);
}

// sum over nu in dirs, nu != mu, of
//   U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
// SEL: the neighbour x+mu by selects on the geometry instead of indexing it
// (kernels whose geometry sits in a parameter struct would copy it to local
// memory to index it).
template <typename R, bool SEL = false>
__device__ __forceinline__ M3<R> staple_sum(const typename vec2<R>::type* __restrict__ U,
                                            const GeomArgs& g, int s, const int c[4], int mu,
                                            unsigned dirs) {
  const long long V = g.V;
  M3<R> C;
  m_zero(C);
  const int s_pmu = SEL ? nb_fwd_rt(g, s, coord_of(c, mu), mu) : nb_fwd(g, s, coord_of(c, mu), mu);
  // not unrolled: one copy of the six products keeps the kernel's hot code
  // small (instruction-fetch stalls dominated the unrolled form)
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu || !((dirs >> nu) & 1u)) continue;
    const int cn = coord_of(c, nu);
    const int Ln = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
    const int sn = nu == 0 ? g.stride[0] : (nu == 1 ? g.stride[1] : (nu == 2 ? g.stride[2] : g.stride[3]));
    const int s_pnu = (cn + 1 < Ln) ? s + sn : s - (Ln - 1) * sn;
    const int s_mnu = (cn > 0) ? s - sn : s + (Ln - 1) * sn;
    const int s_pmu_mnu = (cn > 0) ? s_pmu - sn : s_pmu + (Ln - 1) * sn;
    {
      M3<R> t = mul_nd(ld_link<R>(U, V, mu, s_pnu), ld_link<R>(U, V, nu, s_pmu));
      mac_nn(C, ld_link<R>(U, V, nu, s), t);
    }
    {
      M3<R> t = mul_nn(ld_link<R>(U, V, mu, s_mnu), ld_link<R>(U, V, nu, s_pmu_mnu));
      mac_dn(C, ld_link<R>(U, V, nu, s_mnu), t);
    }
  }
  return C;
}

// Hermitian traceless Q in compact form: real diagonal d0,d1,d2 and the upper
// off-diagonals o01, o02, o12 (Q_kj = conj(Q_jk)).
template <typename R> struct QH {
  R d0, d1, d2;
  cx<R> o01, o02, o12;
};

// the full matrix of a compact Hermitian one
template <typename R>
__device__ __forceinline__ M3<R> qh_full(const QH<R>& q) {
  M3<R> m;
  m.e[0] = mkc<R>(q.d0, 0);
  m.e[4] = mkc<R>(q.d1, 0);
  m.e[8] = mkc<R>(q.d2, 0);
  m.e[1] = q.o01;
  m.e[2] = q.o02;
  m.e[5] = q.o12;
  m.e[3] = cconj(q.o01);
  m.e[6] = cconj(q.o02);
  m.e[7] = cconj(q.o12);
  return m;
}

// Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega)
template <typename R> __device__ __forceinline__ QH<R> q_from_omega(const M3<R>& om) {
  QH<R> q;
  R t = (om.e[0].im + om.e[4].im + om.e[8].im) * R(1.0 / 3.0);
  q.d0 = om.e[0].im - t;
  q.d1 = om.e[4].im - t;
  q.d2 = om.e[8].im - t;
  // Q_jk = (i/2)(conj(Om_kj) - Om_jk) = ((Om_kj.im + Om_jk.im)/2, (Om_kj.re - Om_jk.re)/2)
  q.o01 = mkc<R>(R(0.5) * (om.e[3].im + om.e[1].im), R(0.5) * (om.e[3].re - om.e[1].re));
  q.o02 = mkc<R>(R(0.5) * (om.e[6].im + om.e[2].im), R(0.5) * (om.e[6].re - om.e[2].re));
  q.o12 = mkc<R>(R(0.5) * (om.e[7].im + om.e[5].im), R(0.5) * (om.e[7].re - om.e[5].re));
  return q;
}

template <typename R> __device__ __forceinline__ QH<R> q_rscale(const QH<R>& q, R s) {
  QH<R> r;
  r.d0 = q.d0 * s;
  r.d1 = q.d1 * s;
  r.d2 = q.d2 * s;
  r.o01 = cscale(q.o01, s);
  r.o02 = cscale(q.o02, s);
  r.o12 = cscale(q.o12, s);
  return r;
}

template <typename R> __device__ __forceinline__ R cnorm2(cx<R> a) { return fmaR(a.re, a.re, a.im * a.im); }

// Q^2 of a compact Hermitian Q, again Hermitian (compact).
template <typename R> __device__ __forceinline__ QH<R> q_square(const QH<R>& q) {
  QH<R> r;
  const R n01 = cnorm2(q.o01), n02 = cnorm2(q.o02), n12 = cnorm2(q.o12);
  r.d0 = fmaR(q.d0, q.d0, n01 + n02);
  r.d1 = fmaR(q.d1, q.d1, n01 + n12);
  r.d2 = fmaR(q.d2, q.d2, n02 + n12);
  // (Q^2)_01 = Q01 (d0 + d1) + Q02 conj(Q12)
  r.o01 = cfma_nc(q.o02, q.o12, cscale(q.o01, q.d0 + q.d1));
  // (Q^2)_02 = Q02 (d0 + d2) + Q01 Q12
  r.o02 = cfma(q.o01, q.o12, cscale(q.o02, q.d0 + q.d2));
  // (Q^2)_12 = conj(Q01) Q02 + Q12 (d1 + d2)
  r.o12 = cfma_cn(q.o01, q.o02, cscale(q.o12, q.d1 + q.d2));
  return r;
}

// Threshold on c1 below which the Q -> 0 limit f = (1, i, -1/2) is used, and
// |w| at or below which xi0(w) = sin(w)/w uses its Taylor series.
#define LQ_C1_SERIES 1e-28
#define LQ_XI0_SERIES 0.05

struct CHCoef {
  cx<double> f0, f1, f2;
  int k;   // series order K (degree 2K+1) for small |Q|; 0 when the closed form was used
};

// ---- Small |Q|: the Taylor series of exp(iQ) reduced by Cayley-Hamilton ----
// For traceless Hermitian Q, Q^3 = c1 Q + c0, so every power of Q, and any
// polynomial in Q, is x + y Q + z Q^2.  exp(iQ) truncated at degree N is
// evaluated by Horner's rule on that form: R <- R Q + a_n with
// a_n = i^n / n! is (x, y, z) <- (c0 z + a_n, x + c1 z, y).  The truncation
// error of the matrix series is at most rho^(N+1) / (N+1)! with
// rho = |lambda|_max, and lambda_max^2 <= 4 c1 / 3 for a traceless 3x3
// Hermitian matrix.  N = 2K+1 is the smallest odd degree whose bound is
// under the tolerance: c1 <= (3/4) (tol (2K+2)!)^(1/(K+1)).  No term
// cancels, unlike the closed form's h_j / (9u^2 - w^2) as Q -> 0.
// kExpSeriesA[n] = i^n / n! without its factor i for odd n.
static __constant__ double kExpSeriesA[24] = {
    1.0, 1.0, -0.5, -0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
    -0.001388888888888889, -0.0001984126984126984, 2.48015873015873e-05, 2.7557319223985893e-06,
    -2.755731922398589e-07, -2.505210838544172e-08, 2.08767569878681e-09, 1.6059043836821613e-10,
    -1.1470745597729725e-11, -7.647163731819816e-13, 4.779477332387385e-14, 2.8114572543455206e-15,
    -1.5619206968586225e-16, -8.22063524662433e-18, 4.110317623312165e-19, 1.9572941063391263e-20,
    -8.896791392450574e-22, -3.868170170630684e-23};

// IEEE-754 bit pattern of a positive normal double, at compile time; positive
// doubles order like their bit patterns, so c1 is compared on the integer pipe.
constexpr long long dbl_bits(double x) {
  int e = 0;
  while (x >= 2.0) { x *= 0.5; ++e; }
  while (x < 1.0) { x *= 2.0; --e; }
  return ((long long)(e + 1023) << 52) | (long long)((x - 1.0) * 4503599627370496.0);
}

// Largest c1 handled by the series (|lambda| <= 1); above it the closed form.
#define LQ_SERIES_C1_MAX 0.75

// Series order for c1: thresholds (3/4)(tol (2K+2)!)^(1/(K+1)) for K = 1..,
// the c1 below which the first omitted term, |Q|^(2K+2)/(2K+2)! with
// |Q|^2 <= 4 c1 / 3, stays below tol: tol = 1e-10 for the f_j of FP32 links
// (they are rounded to FP32, 6e-8), 1e-17 on FP64 links.  The stout force
// differentiates the series at one order more than the f_j's.
__device__ __forceinline__ int series_order_f32(double c1) {
  const long long b = __double_as_longlong(c1);
  constexpr long long t[5] = {dbl_bits(3.67423461e-05), dbl_bits(0.00312012573), dbl_bits(0.0336079014),
                              dbl_bits(0.153820376), dbl_bits(0.451978133)};
  int K = 1;
#pragma unroll
  for (int i = 0; i < 5; ++i) K += (b > t[i]);
  return K;   // <= 6: K = 6 covers c1 <= 1.0219
}

__device__ __forceinline__ int series_order_f64(double c1) {
  const long long b = __double_as_longlong(c1);
  constexpr long long t[8] = {dbl_bits(1.161895e-08), dbl_bits(1.44823408e-05), dbl_bits(0.000597642391),
                              dbl_bits(0.00612369949), dbl_bits(0.0307929118), dbl_bits(0.102189274),
                              dbl_bits(0.260099018), dbl_bits(0.552627494)};
  int K = 1;
#pragma unroll
  for (int i = 0; i < 8; ++i) K += (b > t[i]);
  return K;   // <= 9: K = 9 covers c1 <= 1.032
}

// f0 + f1 Q + f2 Q^2 = sum_{n <= 2K+1} (iQ)^n / n!  (c1 <= LQ_SERIES_C1_MAX).
template <int KMAX>
__device__ __forceinline__ void expiq_series(double c0, double c1, int K, CHCoef& f) {
  const int N = 2 * K + 1;
  // the three leading Horner steps from R = 0 give (a_{N-2}, a_{N-1}, a_N)
  double xr = 0.0, xi = kExpSeriesA[N - 2];
  double yr = kExpSeriesA[N - 1], yi = 0.0;
  double zr = 0.0, zi = kExpSeriesA[N];
  // rolled over the warp's largest order (lanes of a smaller order sit out
  // the leading pairs): small code, warp-uniform coefficient loads
  const int Kw = __reduce_max_sync(__activemask(), (unsigned)K);
  (void)KMAX;
#pragma unroll 1
  for (int k = Kw - 1; k >= 1; --k) {
    if (k < K) {
      // n = 2k (a_n real), then n = 2k - 1 (a_n imaginary)
      double nxr = fma(zr, c0, kExpSeriesA[2 * k]), nxi = zi * c0;
      double nyr = fma(zr, c1, xr), nyi = fma(zi, c1, xi);
      zr = yr;
      zi = yi;
      xr = nxr;
      xi = nxi;
      yr = nyr;
      yi = nyi;
      nxr = zr * c0;
      nxi = fma(zi, c0, kExpSeriesA[2 * k - 1]);
      nyr = fma(zr, c1, xr);
      nyi = fma(zi, c1, xi);
      zr = yr;
      zi = yi;
      xr = nxr;
      xi = nxi;
      yr = nyr;
      yi = nyi;
    }
  }
  // n = 0
  f.f0 = mkc(fma(zr, c0, 1.0), zi * c0);
  f.f1 = mkc(fma(zr, c1, xr), fma(zi, c1, xi));
  f.f2 = mkc(yr, yi);
  f.k = K;
}

// f_j with b1_j = df_j/dc1 and b2_j = df_j/dc0 from the same series, by
// differentiating each Horner step (forward mode):
//   x' = c0 z + a_n,  dx'/dc0 = c0 dz/dc0 + z,  dx'/dc1 = c0 dz/dc1
//   y' = x + c1 z,    dy'/dc0 = dx/dc0 + c1 dz/dc0,  dy'/dc1 = dx/dc1 + c1 dz/dc1 + z
//   z' = y.
// The c1 derivative is carried as X1 = dx/dc1 + z, which obeys
//   X1' = c0 dz/dc1 + y,  dy'/dc1 = c1 dz/dc1 + X1,
// two FMAs per component instead of a product, an FMA and an addition;
// dx/dc1 = X1 - z at the end.
// Without the series' cancellation-free form the closed-form b_ij lose
// accuracy like 1e-16 / |Q|^4 as Q -> 0.  One more pair of terms than the
// f_j alone keeps b_ij Q^j at FP64 rounding for all c1 <= 3/4.
template <int KMAX>
__device__ __forceinline__ void expiq_series_deriv(double c0, double c1, int K, cx<double> f[3],
                                                   cx<double> b1[3], cx<double> b2[3]) {
  cx<double> x = mkc(0.0, 0.0), y = x, z = x, x0 = x, y0 = x, z0 = x, X1 = x, y1 = x, z1 = x;
#pragma unroll
  for (int n = 2 * KMAX + 1; n >= 0; --n) {
    if (n <= 2 * K + 1) {
      const cx<double> a = (n & 1) ? mkc(0.0, kExpSeriesA[n]) : mkc(kExpSeriesA[n], 0.0);
      const cx<double> nx = mkc(fma(z.re, c0, a.re), fma(z.im, c0, a.im));
      const cx<double> nx0 = mkc(fma(z0.re, c0, z.re), fma(z0.im, c0, z.im));
      const cx<double> nX1 = mkc(fma(z1.re, c0, y.re), fma(z1.im, c0, y.im));
      const cx<double> ny = mkc(fma(z.re, c1, x.re), fma(z.im, c1, x.im));
      const cx<double> ny0 = mkc(fma(z0.re, c1, x0.re), fma(z0.im, c1, x0.im));
      const cx<double> ny1 = mkc(fma(z1.re, c1, X1.re), fma(z1.im, c1, X1.im));
      z = y;
      z0 = y0;
      z1 = y1;
      x = nx;
      x0 = nx0;
      X1 = nX1;
      y = ny;
      y0 = ny0;
      y1 = ny1;
    }
  }
  f[0] = x;
  f[1] = y;
  f[2] = z;
  b1[0] = mkc(X1.re - z.re, X1.im - z.im);
  b1[1] = y1;
  b1[2] = z1;
  b2[0] = x0;
  b2[1] = y0;
  b2[2] = z0;
}

// c1 = tr(Q^2)/2 and c0 = det Q of the Hermitian Q with diagonal (d0, d1, d2)
// and upper off-diagonal entries o01, o02, o12.  Q is traceless up to the
// rounding of its diagonal; taking d2 = -(d0 + d1) makes it exactly traceless
// in FP64 (the sum of two FP32 entries is exact, that of two FP64 entries
// rounds once), so only d0 and d1 enter:
//   c1 = d0 (d0 + d1) + d1^2 + |o01|^2 + |o02|^2 + |o12|^2
//   c0 = -d0 d1 (d0 + d1) - d0 |o12|^2 - d1 |o02|^2 + (d0 + d1) |o01|^2 + 2 Re(o01 o12 conj(o02))
// (35 flops).  The FMAs are explicit: a sum of two products left to the
// compiler may be fused either way, and differently in different kernels.
__device__ __forceinline__ void ch_invariants(double d0, double d1, cx<double> o01, cx<double> o02, cx<double> o12,
                                              double& c0, double& c1) {
  const double s01 = d0 + d1;   // -d2
  const double n01 = cnorm2(o01), n02 = cnorm2(o02), n12 = cnorm2(o12);
  c1 = fma(d0, s01, fma(d1, d1, n01)) + n02 + n12;
  const cx<double> p = cmul(o01, o12);
  const double re3 = fma(p.re, o02.re, p.im * o02.im);
  c0 = fma(2.0, re3, fma(s01, n01, fma(-d1, n02, fma(-d0, n12, -(d0 * d1) * s01))));
}

// Cayley-Hamilton coefficients of exp(iQ) = f0 + f1 Q + f2 Q^2, in FP64
// (Morningstar & Peardon 2004, Sec. III).  Q must be traceless up to
// rounding (the stout step's Q is; lq_expiq removes the trace of its input
// first) and is made exactly traceless in FP64 by taking d2 = -(d0 + d1)
// (ch_invariants).  For c1 <= 3/4 (all |lambda| <= 1, every link of
// a smearing run on fields with plaquette >~ 0.5) the reduced Taylor series
// above; otherwise the paper's closed form, its quantities formed with few
// FP64 instructions (fp64_math.cuh):
//   1/sqrt(c1/3) by Newton;  |c0|/c0max = |c0| (1/sqrt(c1/3))^3 / 2;
//   cos(theta/3) as the root of 4y^3 - 3y = |c0|/c0max;  w^2 = c1 (1 - y^2);
//   cos w and xi0(w) = sin(w)/w from w^2 by their series when w <= pi/4.
template <int NR = 2>
__device__ __forceinline__ CHCoef ch_coefficients(double d0, double d1, double d2, cx<double> o01,
                                                  cx<double> o02, cx<double> o12) {
  CHCoef f;
  double c0, c1;
  ch_invariants(d0, d1, o01, o02, o12, c0, c1);
  (void)d2;
  if (__double_as_longlong(c1) <= dbl_bits(LQ_SERIES_C1_MAX)) {  // c1 >= +0: integer compare
    expiq_series<NR == 1 ? 6 : 9>(c0, c1, NR == 1 ? series_order_f32(c1) : series_order_f64(c1), f);
    return f;
  }
  f.k = 0;
  if (!(c1 >= LQ_C1_SERIES)) {  // NaN (small c1 took the series)
    f.f0 = mkc(1.0, 0.0);
    f.f1 = mkc(0.0, 1.0);
    f.f2 = mkc(-0.5, 0.0);
    return f;
  }
  const bool neg = c0 < 0.0;
  const double a = c1 * (1.0 / 3.0);
  const double r3 = rsqrt_nr<NR>(a);                               // 1/sqrt(c1/3)
  const double s3 = a * r3;                                        // sqrt(c1/3)
  const double x = fmin(0.5 * fabs(c0) * (r3 * r3 * r3), 1.0);     // |c0| / c0max
  const double y = cos_third_acos<NR>(x);                          // cos(theta/3)
  const double u = s3 * y;
  const double u2 = u * u;
  const double w2 = fmax(c1 * ((1.0 - y) * (1.0 + y)), 0.0);       // w^2 = c1 sin^2(theta/3)
  double cw, xi0;
  if (w2 <= 0.61685027506808491) {                                 // w <= pi/4
    cos_sinc_from_sq(w2, &cw, &xi0);
  } else {
    const double rw = rsqrt_nr<NR>(w2);
    double sw;
    sincos_red(w2 * rw, &sw, &cw);
    xi0 = sw * rw;
  }
  double su, cu;
  sincos_red(u, &su, &cu);
  const cx<double> emiu = mkc(cu, -su);
  const cx<double> e2iu = mkc(fma(cu, cu, -su * su), 2.0 * su * cu);
  // h0 = (u^2 - w^2) e^{2iu} + e^{-iu} [8u^2 cos w + 2iu(3u^2 + w^2) xi0]
  const cx<double> h0 = cadd(cscale(e2iu, u2 - w2),
                             cmul(emiu, mkc(8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0)));
  // h1 = 2u e^{2iu} - e^{-iu} [2u cos w - i(3u^2 - w^2) xi0]
  const cx<double> h1 = csub(cscale(e2iu, 2.0 * u), cmul(emiu, mkc(2.0 * u * cw, -(3.0 * u2 - w2) * xi0)));
  // h2 = e^{2iu} - e^{-iu} [cos w + 3iu xi0]
  const cx<double> h2 = csub(e2iu, cmul(emiu, mkc(cw, 3.0 * u * xi0)));
  const double inv = rcp_nr<NR>(9.0 * u2 - w2);   // 9u^2 - w^2 >= 2 c1 > 0
  f.f0 = cscale(h0, inv);
  f.f1 = cscale(h1, inv);
  f.f2 = cscale(h2, inv);
  if (neg) {  // f_j(-c0) = (-1)^j conj(f_j(c0))
    f.f0 = cconj(f.f0);
    f.f1 = mkc(-f.f1.re, f.f1.im);
    f.f2 = cconj(f.f2);
  }
  return f;
}

// f_j and their derivatives b1_j = df_j/dc1, b2_j = df_j/dc0 (FP64), for the
// stout force (Morningstar & Peardon 2004, Sec. IV).  For c1 <= 3/4 from the
// differentiated series (expiq_series_deriv); otherwise the closed form:  With c1 = 3u^2 + w^2,
// c0 = 2u(u^2 - w^2) and D = 9u^2 - w^2 the chain rule through (u, w) gives
//   b1_j = [2u r1_j + (3u^2 - w^2) r2_j - 2(15u^2 + w^2) f_j] / (2 D^2)
//   b2_j = [r1_j - 3u r2_j - 24u f_j] / (2 D^2)
// with r1_j = dh_j/du and r2_j = (1/w) dh_j/dw, xi1(w) = cos w/w^2 - sin w/w^3.
struct CHDeriv {
  cx<double> f[3], b1[3], b2[3];
};
template <int NR = 2>
__device__ __forceinline__ CHDeriv ch_coefficients_deriv(double d0, double d1, double d2, cx<double> o01,
                                                         cx<double> o02, cx<double> o12) {
  CHDeriv r;
  double c0, c1;
  ch_invariants(d0, d1, o01, o02, o12, c0, c1);
  (void)d2;
  if (__double_as_longlong(c1) <= dbl_bits(LQ_SERIES_C1_MAX)) {
    // The order of the f_j's series plus one.  FP64 links: this keeps b_ij Q^j
    // at FP64 rounding.  FP32 links: the truncated derivatives enter
    // d exp(iQ) = sum_j (b1_j dc1 + b2_j dc0) Q^j + f_j dQ^j with an error
    // <= 2.4e-12 |dQ| over the whole series domain (dc1 ~ 2|Q||dQ|,
    // dc0 ~ 3|Q|^2 |dQ|), far below the FP32 rounding of the links' gradient.
    expiq_series_deriv<10>(c0, c1, (NR == 1 ? series_order_f32(c1) : series_order_f64(c1)) + 1, r.f, r.b1, r.b2);
    return r;
  }
  if (!(c1 >= LQ_C1_SERIES)) {  // NaN (small c1 took the series)
    // Q -> 0: exp(iQ) = 1 + iQ - Q^2/2 - iQ^3/6 + Q^4/24 + iQ^5/120 ... reduced
    // with Q^3 = c1 Q + c0 gives these first derivatives at Q = 0.
    r.f[0] = mkc(1.0, 0.0);
    r.f[1] = mkc(0.0, 1.0);
    r.f[2] = mkc(-0.5, 0.0);
    r.b1[0] = mkc(0.0, 0.0);
    r.b1[1] = mkc(0.0, -1.0 / 6.0);
    r.b1[2] = mkc(1.0 / 24.0, 0.0);
    r.b2[0] = mkc(0.0, -1.0 / 6.0);
    r.b2[1] = mkc(1.0 / 24.0, 0.0);
    r.b2[2] = mkc(0.0, 1.0 / 120.0);
    return r;
  }
  const bool neg = c0 < 0.0;
  // same reductions as ch_coefficients (fp64_math.cuh)
  const double a = c1 * (1.0 / 3.0);
  const double r3 = rsqrt_nr<NR>(a);
  const double s3 = a * r3;
  const double x = fmin(0.5 * fabs(c0) * (r3 * r3 * r3), 1.0);
  const double y = cos_third_acos<NR>(x);
  const double u = s3 * y;
  const double u2 = u * u;
  const double w2 = fmax(c1 * ((1.0 - y) * (1.0 + y)), 0.0);
  double cw, xi0, xi1;
  if (w2 <= 0.61685027506808491) {  // w <= pi/4
    cos_sinc_from_sq(w2, &cw, &xi0);
    xi1 = xi1_from_sq(w2);
  } else {
    const double rw = rsqrt_nr<NR>(w2);
    double sw;
    sincos_red(w2 * rw, &sw, &cw);
    xi0 = sw * rw;
    xi1 = (cw - xi0) * (rw * rw);
  }
  double su, cu;
  sincos_red(u, &su, &cu);
  const cx<double> emiu = mkc(cu, -su);
  const cx<double> e2iu = mkc(fma(cu, cu, -su * su), 2.0 * su * cu);
  const cx<double> I = mkc(0.0, 1.0);
  cx<double> h[3], r1[3], r2[3];
  h[0] = cadd(cscale(e2iu, u2 - w2), cmul(emiu, mkc(8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0)));
  h[1] = csub(cscale(e2iu, 2.0 * u), cmul(emiu, mkc(2.0 * u * cw, -(3.0 * u2 - w2) * xi0)));
  h[2] = csub(e2iu, cmul(emiu, mkc(cw, 3.0 * u * xi0)));
  // r1_0 = 2(u + i(u^2 - w^2)) e^{2iu} + 2 e^{-iu} [4u(2 - iu) cos w + (u(3u^2 + w^2) + i(9u^2 + w^2)) xi0]
  r1[0] = cadd(cmul(mkc(2.0 * u, 2.0 * (u2 - w2)), e2iu),
               cscale(cmul(emiu, mkc(8.0 * u * cw + u * (3.0 * u2 + w2) * xi0,
                                     -4.0 * u2 * cw + (9.0 * u2 + w2) * xi0)), 2.0));
  // r1_1 = 2(1 + 2iu) e^{2iu} + e^{-iu} [-2(1 - iu) cos w + (3u^2 - w^2 + 6iu) xi0]
  r1[1] = cadd(cmul(mkc(2.0, 4.0 * u), e2iu),
               cmul(emiu, mkc(-2.0 * cw + (3.0 * u2 - w2) * xi0, 2.0 * u * cw + 6.0 * u * xi0)));
  // r1_2 = 2i e^{2iu} + i e^{-iu} [cos w - 3(1 - iu) xi0]
  r1[2] = cadd(cmul(mkc(0.0, 2.0), e2iu), cmul(I, cmul(emiu, mkc(cw - 3.0 * xi0, 3.0 * u * xi0))));
  // r2_0 = -2 e^{2iu} + 2iu e^{-iu} [cos w + (1 + 4iu) xi0 + 3u^2 xi1]
  r2[0] = cadd(cscale(e2iu, -2.0),
               cmul(mkc(0.0, 2.0 * u), cmul(emiu, mkc(cw + xi0 + 3.0 * u2 * xi1, 4.0 * u * xi0))));
  // r2_1 = -i e^{-iu} [cos w + (1 + 2iu) xi0 - 3u^2 xi1]
  r2[1] = cmul(mkc(0.0, -1.0), cmul(emiu, mkc(cw + xi0 - 3.0 * u2 * xi1, 2.0 * u * xi0)));
  // r2_2 = e^{-iu} [xi0 - 3iu xi1]
  r2[2] = cmul(emiu, mkc(xi0, -3.0 * u * xi1));
  const double D = 9.0 * u2 - w2;
  const double inv = rcp_nr<NR>(D);
  const double inv2 = 0.5 * inv * inv;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r.f[j] = cscale(h[j], inv);
    r.b1[j] = cscale(csub(cadd(cscale(r1[j], 2.0 * u), cscale(r2[j], 3.0 * u2 - w2)),
                          cscale(r.f[j], 2.0 * (15.0 * u2 + w2))),
                     inv2);
    r.b2[j] = cscale(csub(csub(r1[j], cscale(r2[j], 3.0 * u)), cscale(r.f[j], 24.0 * u)), inv2);
  }
  if (neg) {  // f_j -> (-1)^j conj f_j,  b_ij -> (-1)^(i+j+1) conj b_ij
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double sf = (j % 2 == 0) ? 1.0 : -1.0;
      r.f[j] = cscale(cconj(r.f[j]), sf);
      r.b1[j] = cscale(cconj(r.b1[j]), sf);
      r.b2[j] = cscale(cconj(r.b2[j]), -sf);
    }
  }
  return r;
}

// exp(iQ) = f0 + f1 Q + f2 Q^2 as a full matrix.
template <typename R>
__device__ __forceinline__ M3<R> expiq_assemble(const QH<R>& q, const QH<R>& q2, cx<R> f0, cx<R> f1,
                                                cx<R> f2) {
  M3<R> e;
  e.e[0] = cadd(f0, mkc(fmaR(f2.re, q2.d0, f1.re * q.d0), fmaR(f2.im, q2.d0, f1.im * q.d0)));
  e.e[4] = cadd(f0, mkc(fmaR(f2.re, q2.d1, f1.re * q.d1), fmaR(f2.im, q2.d1, f1.im * q.d1)));
  e.e[8] = cadd(f0, mkc(fmaR(f2.re, q2.d2, f1.re * q.d2), fmaR(f2.im, q2.d2, f1.im * q.d2)));
  e.e[1] = cfma(f2, q2.o01, cmul(f1, q.o01));
  e.e[2] = cfma(f2, q2.o02, cmul(f1, q.o02));
  e.e[5] = cfma(f2, q2.o12, cmul(f1, q.o12));
  e.e[3] = cfma(f2, cconj(q2.o01), cmul(f1, cconj(q.o01)));
  e.e[6] = cfma(f2, cconj(q2.o02), cmul(f1, cconj(q.o02)));
  e.e[7] = cfma(f2, cconj(q2.o12), cmul(f1, cconj(q.o12)));
  return e;
}

// SU(3) re-projection in FP64: Gram-Schmidt of rows 0 and 1, row 2 = conj(row0 x row1).
// Written as FMA chains (norms, row1 - p row0, the cross product) to keep
// the FP64 instruction count low.
// |row|^2 - 1, as an FMA chain started from -1.
__device__ __forceinline__ double row_norm2_m1(const cx<double>* r) {
  double n = fma(r[0].re, r[0].re, -1.0);
  n = fma(r[0].im, r[0].im, n);
  n = fma(r[1].re, r[1].re, n);
  n = fma(r[1].im, r[1].im, n);
  n = fma(r[2].re, r[2].re, n);
  return fma(r[2].im, r[2].im, n);
}

// 1/sqrt(1 + d).  The rows of a link that is unitary to FP32 rounding have
// |d| ~ 1e-7; for |d| <= 2^-16 the Taylor polynomial 1 - d/2 + 3d^2/8
// (- 5d^3/16) is exact to 5|d|^3/16 < 1.2e-15 (to 35 d^4/128 < 1.5e-20 with
// the cubic term, NR >= 2): two or three FMAs instead of a Newton iteration.
// Larger |d| (a far from unitary input) takes the Newton path.
template <int NR> __device__ __forceinline__ double rsqrt_1p(double d) {
  if ((__double_as_longlong(d) & 0x7fffffffffffffffLL) <= dbl_bits(1.52587890625e-05)) {
    if (NR == 1) return fma(d, fma(d, 0.375, -0.5), 1.0);
    return fma(d, fma(d, fma(d, -0.3125, 0.375), -0.5), 1.0);
  }
  return rsqrt_nr<NR>(1.0 + d);
}

template <int NR = 2> __device__ __forceinline__ void reproject_f64(M3<double>& m) {
  const double r0 = rsqrt_1p<NR>(row_norm2_m1(&m.e[0]));
#pragma unroll
  for (int k = 0; k < 3; ++k) m.e[k] = cscale(m.e[k], r0);
  // p = sum_k conj(row0_k) row1_k;  row1 <- row1 - p row0
  cx<double> p = mkc(m.e[0].re * m.e[3].re, m.e[0].re * m.e[3].im);
  p.re = fma(m.e[0].im, m.e[3].im, p.re);
  p.im = fma(-m.e[0].im, m.e[3].re, p.im);
  p = cfma_cn(m.e[1], m.e[4], p);
  p = cfma_cn(m.e[2], m.e[5], p);
  const cx<double> mp = mkc(-p.re, -p.im);
#pragma unroll
  for (int k = 0; k < 3; ++k) m.e[3 + k] = cfma(mp, m.e[k], m.e[3 + k]);
  const double r1 = rsqrt_1p<NR>(row_norm2_m1(&m.e[3]));
#pragma unroll
  for (int k = 0; k < 3; ++k) m.e[3 + k] = cscale(m.e[3 + k], r1);
  // row2 = conj(row0 x row1), each entry a*b - c*d as one product and one complex FMA
  auto cross = [&](int a, int b, int c, int d) {
    const cx<double> t = cmul(m.e[c], m.e[d]);
    return cconj(cfma(m.e[a], m.e[b], mkc(-t.re, -t.im)));
  };
  m.e[6] = cross(1, 5, 2, 4);
  m.e[7] = cross(2, 3, 0, 5);
  m.e[8] = cross(0, 4, 1, 3);
}

template <typename A, typename B> __device__ __forceinline__ M3<A> m_convert(const M3<B>& m) {
  M3<A> r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = mkc<A>((A)m.e[i].re, (A)m.e[i].im);
  return r;
}
// FP32 <-> FP64 element conversions on the integer pipe (fp64_math.cuh).
__device__ __forceinline__ double to_f64(float x) { return f2d(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return d2f(x); }
template <typename R> __device__ __forceinline__ R from_f64(double x);
template <> __device__ __forceinline__ float from_f64<float>(double x) { return d2f(x); }
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }

// Re-projects a link held in precision R through FP64 (rows 0 and 1 are
// converted in, all three rows converted out).
template <typename R> __device__ __forceinline__ M3<R> reproject_via_f64(const M3<R>& m) {
  M3<double> d;
#pragma unroll
  for (int i = 0; i < 6; ++i) d.e[i] = mkc(to_f64(m.e[i].re), to_f64(m.e[i].im));
  reproject_f64<sizeof(R) == 4 ? 1 : 2>(d);
  M3<R> r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = mkc<R>(from_f64<R>(d.e[i].re), from_f64<R>(d.e[i].im));
  return r;
}

// The FP64 re-projection of an FP32 link, arranged so that the FP64 pipe does
// only the cancellation-prone part.  Rows u0, u1 of the FP32 link are exact
// in FP64 and so are the products of their entries; Gram-Schmidt gives
//   r0 = n0 u0,  r1 = n1 (u1 - c u0),  r2 = conj(r0 x r1),
//   n0 = (1 + d0)^(-1/2),  d0 = |u0|^2 - 1,  p = u0^dag u1,  c = n0^2 p,
//   n1 = (1 + d1)^(-1/2),  d1 = |u1|^2 - 1 - n0^2 |p|^2.
// d0, |u1|^2 - 1 and p (sums that cancel to ~1e-7) and the cross product
// u0 x u1 (entries that can be small) are formed in FP64.  For a link unitary
// to FP32 rounding the rest are corrections of relative size <= 2^-16
// (checked; otherwise the Gram-Schmidt of reproject_f64 runs on the whole
// link), so their FP32 rounding (6e-8 of a correction) stays below 1e-12:
//   row 0  = u0 + e0 u0,           e0 = n0 - 1 = -d0/2 + 3 d0^2/8
//   row 1  = u1 + a1,              a1 = e1 u1 - c n1 u0,  e1 = n1 - 1
//   r0 x r1 = u0 x u1 + e0 (u0 x u1) + n0 (u0 x a1)   (products of two corrections dropped)
// each row rounded to FP32 once, the FP32 correction of row 2 folded into the
// accumulator of its FP64 cross product.  The result is the FP64 Gram-Schmidt
// rounded to FP32 except where the exact value lies within ~1e-12 of a
// rounding boundary; 48 FP64 instructions against 76.
static __device__ __noinline__ M3<float> reproject_f32_general(M3<float> m) {
  M3<double> d;
#pragma unroll
  for (int i = 0; i < 6; ++i) d.e[i] = mkc(to_f64(m.e[i].re), to_f64(m.e[i].im));
  reproject_f64<1>(d);
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = mkc<float>(from_f64<float>(d.e[i].re), from_f64<float>(d.e[i].im));
  return m;
}

__device__ __forceinline__ M3<float> reproject_f32(const M3<float>& m) {
  cx<double> r[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) r[i] = mkc(to_f64(m.e[i].re), to_f64(m.e[i].im));
  const double d0 = row_norm2_m1(&r[0]);
  const double d1b = row_norm2_m1(&r[3]);
  cx<double> p = mkc(r[0].re * r[3].re, r[0].re * r[3].im);   // sum_k conj(u0_k) u1_k
  p.re = fma(r[0].im, r[3].im, p.re);
  p.im = fma(-r[0].im, r[3].re, p.im);
  p = cfma_cn(r[1], r[4], p);
  p = cfma_cn(r[2], r[5], p);
  const float d0f = to_f32(d0), d1bf = to_f32(d1b);
  const cx<float> pf = mkc(to_f32(p.re), to_f32(p.im));
  const float lim = 1.52587890625e-05f;   // 2^-16
  if (!(fabsf(d0f) <= lim && fabsf(d1bf) <= lim && fabsf(pf.re) + fabsf(pf.im) <= lim))
    return reproject_f32_general(m);
  const float e0 = d0f * fmaf(d0f, 0.375f, -0.5f);
  const float n0sq = fmaf(2.0f, e0, 1.0f);                    // (1 + e0)^2 up to e0^2
  const float d1f = fmaf(-n0sq, fmaf(pf.re, pf.re, pf.im * pf.im), d1bf);
  const float e1 = d1f * fmaf(d1f, 0.375f, -0.5f);
  const float cs = n0sq * (1.0f + e1);                         // c n1 = n0^2 n1 p
  const cx<float> cn = mkc(pf.re * cs, pf.im * cs);
  M3<float> out;
  cx<float> a1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cx<float> u0 = m.e[k], u1 = m.e[3 + k];
    out.e[k] = mkc(fmaf(u0.re, e0, u0.re), fmaf(u0.im, e0, u0.im));
    // a1 = e1 u1 - cn u0
    a1[k] = mkc(fmaf(-cn.re, u0.re, fmaf(cn.im, u0.im, e1 * u1.re)),
                fmaf(-cn.re, u0.im, fmaf(-cn.im, u0.re, e1 * u1.im)));
    out.e[3 + k] = mkc(u1.re + a1[k].re, u1.im + a1[k].im);
  }
  const float n0 = 1.0f + e0;
  // component j of r0 x r1: (i, l) the two other indices, r0_i r1_l - r0_l r1_i
  auto row2 = [&](int i, int l) {
    const cx<float> u0i = m.e[i], u0l = m.e[l], u1i = m.e[3 + i], u1l = m.e[3 + l];
    const cx<float> x = csub(cmul(u0i, u1l), cmul(u0l, u1i));             // u0 x u1 (FP32 copy)
    const cx<float> y = csub(cmul(u0i, a1[l]), cmul(u0l, a1[i]));         // u0 x a1
    const cx<float> corr = mkc(fmaf(e0, x.re, n0 * y.re), fmaf(e0, x.im, n0 * y.im));
    // FP64: u0_i u1_l - (u0_l u1_i - corr)
    const cx<double> t = cfma(r[l], r[3 + i], mkc(-to_f64(corr.re), -to_f64(corr.im)));
    const cx<double> v = cfma(r[i], r[3 + l], mkc(-t.re, -t.im));
    return mkc(to_f32(v.re), -to_f32(v.im));
  };
  out.e[6] = row2(1, 2);
  out.e[7] = row2(2, 0);
  out.e[8] = row2(0, 1);
  return out;
}

template <typename R> __device__ __forceinline__ M3<R> reproject_link(const M3<R>& m) { return reproject_via_f64(m); }
template <> __device__ __forceinline__ M3<float> reproject_link<float>(const M3<float>& m) { return reproject_f32(m); }

// New link from the bare staple sum S and U_mu(x): FP64 coefficients always;
// matrix algebra in R; optional FP64 re-projection.
template <typename R>
__device__ __forceinline__ M3<R> stout_update(const M3<R>& S, const M3<R>& Umu, R rho, bool reproject,
                                              int* korder = nullptr) {
  // Q is linear in Omega = rho S U^dag: scale the 9 real components of Q
  // instead of the 18 of the staple sum
  const QH<R> q = q_rscale(q_from_omega(mul_nd(S, Umu)), rho);
  // FP32 links: one Newton step per FP64 refinement (~1e-13); FP64 links: two
  const CHCoef f = ch_coefficients<sizeof(R) == 4 ? 1 : 2>(to_f64(q.d0), to_f64(q.d1), to_f64(q.d2),
                                   mkc(to_f64(q.o01.re), to_f64(q.o01.im)), mkc(to_f64(q.o02.re), to_f64(q.o02.im)),
                                   mkc(to_f64(q.o12.re), to_f64(q.o12.im)));
  const QH<R> q2 = q_square(q);
  const M3<R> E = expiq_assemble(q, q2, mkc<R>(from_f64<R>(f.f0.re), from_f64<R>(f.f0.im)),
                                 mkc<R>(from_f64<R>(f.f1.re), from_f64<R>(f.f1.im)),
                                 mkc<R>(from_f64<R>(f.f2.re), from_f64<R>(f.f2.im)));
  M3<R> Up = mul_nn(E, Umu);
  if (reproject) Up = reproject_link<R>(Up);
  if (korder) *korder = f.k;
  return Up;
}

// New link U'_mu(x) for one (site, mu), neighbours read from global memory.
template <typename R>
__device__ __forceinline__ M3<R> stout_link(const typename vec2<R>::type* __restrict__ U,
                                            const GeomArgs& g, int s, const int c[4], int mu,
                                            unsigned dirs, R rho, bool reproject, int* korder = nullptr) {
  return stout_update<R>(staple_sum<R>(U, g, s, c, mu, dirs), ld_link<R>(U, g.V, mu, s), rho, reproject,
                         korder);
}

}  // namespace lq
