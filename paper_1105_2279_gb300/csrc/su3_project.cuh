// SU(3) projection shared by the APE and HYP kernels: the unitary polar
// factor with the determinant phase removed,
//   W = V (V^dag V)^(-1/2),   P(V) = W exp(-i arg(det W) / 3),   arg in (-pi, pi],
// in FP64.  (V^dag V)^(-1/2): A = V^dag V is Hermitian positive definite with
// eigenvalues l1, l2, l3 (the trigonometric roots of its characteristic
// cubic, cos(theta/3) from fp64_math.cuh), and for any f,
//   f(A) = f[l1] + f[l1,l2] (A - l1) + f[l1,l2,l3] (A - l1)(A - l2)
// (Newton's interpolation of f on the spectrum; Cayley-Hamilton).  For
// f(x) = x^(-1/2) and s_k = sqrt(l_k) the divided differences are
//   f[l1,l2] = -1 / (s1 s2 (s1 + s2)),
//   f[l1,l2,l3] = (s1 + s2 + s3) / (s1 s2 s3 (s1 + s2)(s2 + s3)(s1 + s3)),
// free of cancellation, so degenerate spectra need no special case.
// det W = det V / |det V|, so arg(det W) = arg(det V).  Square roots,
// reciprocals and the cube root of the determinant phase come from FP32 seeds
// and FP64 Newton steps, no library calls.  V's singular values must lie in
// FP32's normal range.
#pragma once

#include "stout_core.cuh"

namespace lq {

// Unitary polar factor of a non-singular V by the scaled Newton iteration
// (at most 16 steps; it stops once a step moves no entry by more than 1e-15).
static __device__ __noinline__ M3<double> polar_newton(M3<double> y) {
#pragma unroll 1
  for (int it = 0; it < 16; ++it) {
    // adjugate: adj(Y)_ij = cofactor_ji
    M3<double> ad;
    ad.e[0] = csub(cmul(y.e[4], y.e[8]), cmul(y.e[5], y.e[7]));
    ad.e[1] = csub(cmul(y.e[2], y.e[7]), cmul(y.e[1], y.e[8]));
    ad.e[2] = csub(cmul(y.e[1], y.e[5]), cmul(y.e[2], y.e[4]));
    ad.e[3] = csub(cmul(y.e[5], y.e[6]), cmul(y.e[3], y.e[8]));
    ad.e[4] = csub(cmul(y.e[0], y.e[8]), cmul(y.e[2], y.e[6]));
    ad.e[5] = csub(cmul(y.e[2], y.e[3]), cmul(y.e[0], y.e[5]));
    ad.e[6] = csub(cmul(y.e[3], y.e[7]), cmul(y.e[4], y.e[6]));
    ad.e[7] = csub(cmul(y.e[1], y.e[6]), cmul(y.e[0], y.e[7]));
    ad.e[8] = csub(cmul(y.e[0], y.e[4]), cmul(y.e[1], y.e[3]));
    const cx<double> det = cadd(cadd(cmul(y.e[0], ad.e[0]), cmul(y.e[1], ad.e[3])), cmul(y.e[2], ad.e[6]));
    // Y^(-dag) = adj(Y)^dag / conj(det) = adj(Y)^dag det / |det|^2
    const double idn = 1.0 / cnorm2(det);
    double ny = 0.0, ni = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      ny += cnorm2(y.e[i]);
      ni += cnorm2(ad.e[i]);
    }
    ni *= idn;                                 // |Y^(-1)|_F^2
    const double zeta = sqrt(sqrt(ni / ny));   // sqrt(|Y^-1|_F / |Y|_F)
    double move = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<double> a = cconj(ad.e[3 * k + i]);   // (adj Y)^dag_ik
        const cx<double> inv = mkc((a.re * det.re - a.im * det.im) * idn, (a.re * det.im + a.im * det.re) * idn);
        const cx<double> old = y.e[3 * i + k];
        const cx<double> nw = mkc(0.5 * (zeta * old.re + inv.re / zeta), 0.5 * (zeta * old.im + inv.im / zeta));
        move = fmax(move, fabs(nw.re - old.re) + fabs(nw.im - old.im));
        y.e[3 * i + k] = nw;
      }
    if (move < 1e-15) break;
  }
  return y;
}

// The pieces of P(V) = W z: the polar factor W, the phase z = exp(-i arg(det V) / 3),
// A = V^dag V (compact Hermitian) and |det V| (= det (V^dag V)^(1/2)).
struct PolarParts {
  M3<double> W;
  cx<double> z;
  QH<double> A;
  double absdet;
};

// NR: Newton steps after the FP32 seeds of the square roots, reciprocals and
// the cube root (1 on FP32 links, ~1e-13 relative; 2 on FP64 links).
template <int NR>
__device__ __forceinline__ PolarParts polar_parts_f64(const M3<double>& v) {
  // A = V^dag V: A_ij = sum_k conj(V_ki) V_kj
  double a00 = 0, a11 = 0, a22 = 0;
  cx<double> a01 = mkc(0.0, 0.0), a02 = a01, a12 = a01;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cx<double> v0 = v.e[3 * k], v1 = v.e[3 * k + 1], v2 = v.e[3 * k + 2];
    a00 = fma(v0.re, v0.re, fma(v0.im, v0.im, a00));
    a11 = fma(v1.re, v1.re, fma(v1.im, v1.im, a11));
    a22 = fma(v2.re, v2.re, fma(v2.im, v2.im, a22));
    a01 = cfma_cn(v0, v1, a01);
    a02 = cfma_cn(v0, v2, a02);
    a12 = cfma_cn(v1, v2, a12);
  }
  // eigenvalues: A = m + B with B traceless; B's roots 2 sqrt(p) cos(theta/3 + 2 pi k/3),
  // p = tr(B^2)/6, cos(theta) = q / p^(3/2), q = det(B)/2
  const double m = (a00 + a11 + a22) * (1.0 / 3.0);
  const double b0 = a00 - m, b1 = a11 - m, b2 = a22 - m;
  const double n01 = cnorm2(a01), n02 = cnorm2(a02), n12 = cnorm2(a12);
  const double p = (b0 * b0 + b1 * b1 + b2 * b2) * (1.0 / 6.0) + (n01 + n02 + n12) * (1.0 / 3.0);
  const cx<double> t = cmul(a01, a12);
  const double re3 = t.re * a02.re + t.im * a02.im;   // Re(a01 a12 conj(a02))
  const double q = 0.5 * (b0 * b1 * b2 - b0 * n12 - b1 * n02 - b2 * n01 + 2.0 * re3);
  double sp = 0.0, r = 0.0;
  if (p > 1e-30) {   // below: eigenvalue spread < 1e-15 of the scale, taken as degenerate
    const double rp = rsqrt_nr<NR>(p);
    sp = p * rp;                                         // sqrt(p)
    r = fmin(fabs(q) * (rp * rp * rp), 1.0);             // |q| / p^(3/2)
  }
  const double y = cos_third_acos<NR>(r);
  const double w2 = fmax(1.0 - y * y, 0.0);
  const double z = w2 > 0.0 ? w2 * rsqrt_nr<NR>(w2) : 0.0;  // sqrt(1 - y^2)
  const double sg = q < 0.0 ? -1.0 : 1.0;
  // det V first: |det V|^2 = det A fixes the smallest eigenvalue to full
  // relative precision (the trigonometric roots carry an absolute error of
  // about eps * l_max, too much for l_min << l_max)
  const cx<double> m0 = csub(cmul(v.e[4], v.e[8]), cmul(v.e[5], v.e[7]));
  const cx<double> m1 = csub(cmul(v.e[3], v.e[8]), cmul(v.e[5], v.e[6]));
  const cx<double> m2 = csub(cmul(v.e[3], v.e[7]), cmul(v.e[4], v.e[6]));
  const cx<double> det = cadd(csub(cmul(v.e[0], m0), cmul(v.e[1], m1)), cmul(v.e[2], m2));
  const double detA = cnorm2(det);
  double l1 = m + sg * 2.0 * sp * y;   // the largest for sg > 0, the smallest otherwise
  const double l2 = m + sg * sp * (-y + 1.7320508075688772 * z);
  double l3 = m + sg * sp * (-y - 1.7320508075688772 * z);
  if (sg > 0.0) l3 = detA * rcp_nr<NR>(l1 * l2);
  else l1 = detA * rcp_nr<NR>(l2 * l3);
  const double lmax = sg > 0.0 ? l1 : l3, lmin = sg > 0.0 ? l3 : l1;
  const double r1 = rsqrt_nr<NR>(l1), r2 = rsqrt_nr<NR>(l2), r3 = rsqrt_nr<NR>(l3);   // 1/s_k
  const double s1 = l1 * r1, s2 = l2 * r2, s3 = l3 * r3;
  const double d1 = r1;
  const double s12 = s1 + s2;
  const double d12 = -(r1 * r2) * rcp_nr<NR>(s12);
  const double d123 = (s1 + s2 + s3) * (r1 * r2 * r3) * rcp_nr<NR>(s12 * (s2 + s3) * (s1 + s3));
  // X = d1 + d12 (A - l1) + d123 (A - l1)(A - l2) = c0 + c1 A + c2 A^2
  const double c2 = d123, c1 = d12 - d123 * (l1 + l2), c0 = d1 - d12 * l1 + d123 * l1 * l2;
  // A and A^2 in the compact Hermitian form (real diagonal, upper triangle)
  QH<double> A;
  A.d0 = a00;
  A.d1 = a11;
  A.d2 = a22;
  A.o01 = a01;
  A.o02 = a02;
  A.o12 = a12;
  const QH<double> A2 = q_square(A);
  auto comb = [&](cx<double> a, cx<double> a2) {
    return mkc(fma(c2, a2.re, c1 * a.re), fma(c2, a2.im, c1 * a.im));
  };
  M3<double> X;
  X.e[0] = mkc(fma(c2, A2.d0, fma(c1, A.d0, c0)), 0.0);
  X.e[4] = mkc(fma(c2, A2.d1, fma(c1, A.d1, c0)), 0.0);
  X.e[8] = mkc(fma(c2, A2.d2, fma(c1, A.d2, c0)), 0.0);
  X.e[1] = comb(A.o01, A2.o01);
  X.e[2] = comb(A.o02, A2.o02);
  X.e[5] = comb(A.o12, A2.o12);
  X.e[3] = cconj(X.e[1]);
  X.e[6] = cconj(X.e[2]);
  X.e[7] = cconj(X.e[5]);
  M3<double> W = mul_nn(v, X);
  // The monomial form c0 + c1 A + c2 A^2 loses about eps * l_max / l_min to
  // cancellation.  For l_max / l_min > 1e2 (cond V > 10; rare on smooth
  // fields) the polar factor comes instead from the scaled Newton iteration
  //   Y <- (z Y + Y^(-dag) / z) / 2,   z = sqrt(|Y^(-1)|_F / |Y|_F),   Y_0 = V
  // (N. J. Higham, Functions of Matrices, SIAM 2008, Sec. 8.6), backward
  // stable and independent of the spectrum; Y^(-dag) = adj(Y)^dag / conj(det Y).
  if (lmax > 1e2 * lmin) W = polar_newton(v);
  // exp(-i arg(det V) / 3)
  // e^{-i phi/3}, phi = arg(det V) in (-pi, pi]: the principal cube root w of
  // z = det/|det|, from the FP32 angle phi/3, refined by w <- (2w + z conj(w)^2)/3
  // (Newton for w^3 = z with 1/w^2 = conj(w)^2 on the unit circle): the phase
  // error e becomes O(e^2), the modulus error grows by 4/3 per step and is
  // removed by a final normalisation; then conjugated
  const double ar = rsqrt_nr<NR>(cnorm2(det));
  const cx<double> zz = mkc(det.re * ar, det.im * ar);
  float sf, cf;
  __sincosf(atan2f(d2f(zz.im), d2f(zz.re)) * (1.0f / 3.0f), &sf, &cf);
  cx<double> w = mkc(f2d(cf), f2d(sf));
#pragma unroll
  for (int it = 0; it < NR + 1; ++it) {
    const cx<double> wc = cconj(w);
    const cx<double> t2 = cmul(zz, cmul(wc, wc));
    w = mkc((2.0 * w.re + t2.re) * (1.0 / 3.0), (2.0 * w.im + t2.im) * (1.0 / 3.0));
  }
  const double wn = rsqrt_nr<NR>(cnorm2(w));
  PolarParts pp;
  pp.W = W;
  pp.z = mkc(w.re * wn, -w.im * wn);
  pp.A = A;
  pp.absdet = cnorm2(det) * ar;
  return pp;
}

template <int NR>
__device__ __forceinline__ M3<double> project_su3_f64(const M3<double>& v) {
  const PolarParts pp = polar_parts_f64<NR>(v);
  M3<double> P;
#pragma unroll
  for (int i = 0; i < 9; ++i) P.e[i] = cmul(pp.W.e[i], pp.z);
  return P;
}

// Inverse of a Hermitian matrix from its adjugate (inverse_ij = cofactor_ji / det).
__device__ __forceinline__ QH<double> qh_inverse(const QH<double>& h) {
  const double a = h.d0, d = h.d1, f = h.d2;
  const cx<double> b = h.o01, c = h.o02, e = h.o12;
  QH<double> r;
  r.d0 = d * f - cnorm2(e);
  r.d1 = a * f - cnorm2(c);
  r.d2 = a * d - cnorm2(b);
  r.o01 = csub(cmul(c, cconj(e)), cscale(b, f));
  r.o02 = csub(cmul(b, e), cscale(c, d));
  r.o12 = csub(cmul(c, cconj(b)), cscale(e, a));
  // det = a (d f - |e|^2) - f |b|^2 - d |c|^2 + 2 Re(b e conj(c))
  const cx<double> be = cmul(b, e);
  const double det = a * r.d0 - f * cnorm2(b) - d * cnorm2(c) + 2.0 * (be.re * c.re + be.im * c.im);
  const double id = 1.0 / det;
  r.d0 *= id;
  r.d1 *= id;
  r.d2 *= id;
  r.o01 = cscale(r.o01, id);
  r.o02 = cscale(r.o02, id);
  r.o12 = cscale(r.o12, id);
  return r;
}

// Hermitian part (M + M^dag)/2 in compact form
__device__ __forceinline__ QH<double> herm_part(const M3<double>& m) {
  QH<double> h;
  h.d0 = m.e[0].re;
  h.d1 = m.e[4].re;
  h.d2 = m.e[8].re;
  h.o01 = mkc(0.5 * (m.e[1].re + m.e[3].re), 0.5 * (m.e[1].im - m.e[3].im));
  h.o02 = mkc(0.5 * (m.e[2].re + m.e[6].re), 0.5 * (m.e[2].im - m.e[6].im));
  h.o12 = mkc(0.5 * (m.e[5].re + m.e[7].re), 0.5 * (m.e[5].im - m.e[7].im));
  return h;
}

// Gradient through P: given G_P (G = dS/dRe + i dS/dIm, dS = Re tr(G^dag dP)),
// returns G_V.  With Z = (V^dag V)^(1/2) (so W = V Z^-1) and p1, p2, p3 the
// elementary symmetric functions of Z's eigenvalues s_k:
//   P = W z, z = (det W)^(-1/3), dz = -(z/3) tr(W^dag dW) on the unitary W:
//       G_W = conj(z) G_P + (i/3) Im tr(G_P^dag P) W
//   W = V X, X = Z^-1:  G_V = G_W X + 2 V dX[H],  H = Herm(V^dag G_W),
//       dX[H] the derivative of X = A^(-1/2) along dA = H; dX = -X Y X
//       with Y the solution of the Lyapunov equation Z Y + Y Z = H.
//   The Lyapunov equation in closed form (no eigenvectors): with L, R the
//   left and right multiplications by Z, 1/(x + y) reduces modulo the
//   characteristic polynomial t^3 - p1 t^2 + p2 t - p3 of both to
//     (x^2 - x y + y^2 - p1 x + p1 y + p2) / (2 (p1 y^2 + p3)),
//   so Y = A C + C A - Z C Z - p1 (Z C - C Z) + p2 C with C = H (p1 A + p3)^-1 / 2
//   (A = Z^2).  Its terms carry magnitudes up to s_max^2 |C|, so it loses
//   about s_max / s_min in relative accuracy.
// Then G_V = (G_W - 2 W Y) X.  All FP64.
template <int NR>
__device__ __forceinline__ M3<double> project_su3_vjp_f64(const M3<double>& v, const M3<double>& gp) {
  const PolarParts pp = polar_parts_f64<NR>(v);
  double kim = 0.0;   // Im tr(G_P^dag P) = Im sum conj(G_P) P
  M3<double> gw;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<double> p = cmul(pp.W.e[i], pp.z);
    kim = fma(gp.e[i].re, p.im, fma(-gp.e[i].im, p.re, kim));
  }
  const double k3 = kim * (1.0 / 3.0);
  const cx<double> zc = cconj(pp.z);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<double> a = cmul(zc, gp.e[i]);
    gw.e[i] = mkc(a.re - k3 * pp.W.e[i].im, a.im + k3 * pp.W.e[i].re);
  }
  const QH<double> Zh = herm_part(mul_dn(v, pp.W));
  const double p1 = Zh.d0 + Zh.d1 + Zh.d2;
  const double p2 = 0.5 * (p1 * p1 - (pp.A.d0 + pp.A.d1 + pp.A.d2));
  const double p3 = pp.absdet;
  const M3<double> X = qh_full(qh_inverse(Zh));
  const M3<double> Z = qh_full(Zh), A = qh_full(pp.A);
  QH<double> Bh = pp.A;   // p1 A + p3
  Bh.d0 = fma(p1, Bh.d0, p3);
  Bh.d1 = fma(p1, Bh.d1, p3);
  Bh.d2 = fma(p1, Bh.d2, p3);
  Bh.o01 = cscale(Bh.o01, p1);
  Bh.o02 = cscale(Bh.o02, p1);
  Bh.o12 = cscale(Bh.o12, p1);
  const M3<double> N = qh_full(qh_inverse(Bh));
  const M3<double> C = m_rscale(mul_nn(qh_full(herm_part(mul_dn(v, gw))), N), 0.5);
  const M3<double> ZC = mul_nn(Z, C), CZ = mul_nn(C, Z);
  M3<double> Y = mul_nn(A, C);
  mac_nn(Y, C, A);
  Y = m_sub(Y, mul_nn(ZC, Z));
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<double> d = csub(ZC.e[i], CZ.e[i]);
    Y.e[i] = mkc(fma(p2, C.e[i].re, fma(-p1, d.re, Y.e[i].re)), fma(p2, C.e[i].im, fma(-p1, d.im, Y.e[i].im)));
  }
  const M3<double> Yh = qh_full(herm_part(Y));
  return mul_nn(m_sub(gw, m_rscale(mul_nn(pp.W, Yh), 2.0)), X);
}

}  // namespace lq
