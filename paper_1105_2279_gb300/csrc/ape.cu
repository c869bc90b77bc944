// APE link smearing (M. Albanese et al., Phys. Lett. B 192 (1987) 163), an
// adjacent smearing on the same staple sum as the stout step:
//   V_mu(x) = (1 - alpha) U_mu(x) + alpha / (2 (d - 1)) * C_mu(x),   d = |dirs|,
//   U'_mu(x) = P(V_mu(x)),
// C the staple sum of the stout step (without rho) and P the projection to
// SU(3) by the unitary polar factor with the determinant phase removed:
//   W = V (V^dag V)^(-1/2),   P(V) = W exp(-i arg(det W) / 3),   arg in (-pi, pi].
// The mixing runs in the field precision, P always in FP64: square roots,
// reciprocals and the cube root of the determinant phase from FP32 seeds and
// FP64 Newton steps (fp64_math.cuh), no library calls.
//
// (V^dag V)^(-1/2): A = V^dag V is Hermitian positive definite with
// eigenvalues l1, l2, l3 (the trigonometric roots of its characteristic
// cubic, cos(theta/3) from fp64_math.cuh), and for any f,
//   f(A) = f[l1] + f[l1,l2] (A - l1) + f[l1,l2,l3] (A - l1)(A - l2)
// (Newton's interpolation of f on the spectrum; Cayley-Hamilton).  For
// f(x) = x^(-1/2) and s_k = sqrt(l_k) the divided differences are
//   f[l1,l2] = -1 / (s1 s2 (s1 + s2)),
//   f[l1,l2,l3] = (s1 + s2 + s3) / (s1 s2 s3 (s1 + s2)(s2 + s3)(s1 + s3)),
// free of cancellation, so degenerate spectra need no special case.
// det W = det V / |det V|, so arg(det W) = arg(det V).
#include "lq_internal.h"
#include "stout_core.cuh"

namespace lq {

struct ApeDirs {
  int mu[4];
};

// NR: Newton steps after the FP32 seeds of the square roots, reciprocals and
// the cube root (1 on FP32 links, ~1e-13 relative; 2 on FP64 links).
template <int NR>
__device__ __forceinline__ M3<double> project_su3_f64(const M3<double>& v) {
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
  const double l1 = m + sg * 2.0 * sp * y;
  const double l2 = m + sg * sp * (-y + 1.7320508075688772 * z);
  const double l3 = m + sg * sp * (-y - 1.7320508075688772 * z);
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
  // det V, then exp(-i arg(det V) / 3)
  const cx<double> m0 = csub(cmul(v.e[4], v.e[8]), cmul(v.e[5], v.e[7]));
  const cx<double> m1 = csub(cmul(v.e[3], v.e[8]), cmul(v.e[5], v.e[6]));
  const cx<double> m2 = csub(cmul(v.e[3], v.e[7]), cmul(v.e[4], v.e[6]));
  const cx<double> det = cadd(csub(cmul(v.e[0], m0), cmul(v.e[1], m1)), cmul(v.e[2], m2));
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
  const cx<double> ph = mkc(w.re * wn, -w.im * wn);
#pragma unroll
  for (int i = 0; i < 9; ++i) W.e[i] = cmul(W.e[i], ph);
  return W;
}

template <typename R>
__global__ void __launch_bounds__(256) k_ape(const typename vec2<R>::type* __restrict__ Uin,
                                             typename vec2<R>::type* __restrict__ Uout, GeomArgs g, R keep, R coef,
                                             unsigned dirs, int nd, ApeDirs ad) {
  const int mi = blockIdx.x % nd;
  const long long sl = (long long)(blockIdx.x / nd) * blockDim.x + threadIdx.x;
  const long long V = g.V;
  if (sl >= V) return;
  const int mu = mi == 0 ? ad.mu[0] : (mi == 1 ? ad.mu[1] : (mi == 2 ? ad.mu[2] : ad.mu[3]));
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  const M3<R> C = staple_sum<R>(Uin, g, s, c, mu, dirs);
  const M3<R> U = ld_link<R>(Uin, V, mu, s);
  M3<double> v;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<R> e = mkc<R>(fmaR(coef, C.e[i].re, keep * U.e[i].re), fmaR(coef, C.e[i].im, keep * U.e[i].im));
    v.e[i] = mkc(to_f64(e.re), to_f64(e.im));
  }
  const M3<double> P = project_su3_f64<sizeof(R) == 4 ? 1 : 2>(v);
  M3<R> out;
#pragma unroll
  for (int i = 0; i < 9; ++i) out.e[i] = mkc<R>(from_f64<R>(P.e[i].re), from_f64<R>(P.e[i].im));
  st_m3<R>(Uout + (long long)mu * 9 * V + s, V, out);
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_ape_smear(lq_field* links, double alpha, int n_steps, unsigned dirs_mask, void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_ape_smear");
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_ape_smear")) != LQ_OK) return st;
  if (!(alpha == alpha) || alpha > 1e6 || alpha < -1e6 || n_steps < 0) {
    set_error("lq_ape_smear: alpha must be finite and n_steps >= 0");
    return LQ_ERR_ARG;
  }
  if (n_steps == 0) return LQ_OK;
  cudaStream_t s = as_stream(stream);
  const GeomArgs g = geom_args(links->geom);
  ApeDirs ad;
  int nd = 0;
  for (int mu = 0; mu < 4; ++mu)
    if ((dirs_mask >> mu) & 1u) ad.mu[nd++] = mu;
  for (int j = nd; j < 4; ++j) ad.mu[j] = 0;
  const double coef = nd > 1 ? alpha / (2.0 * (nd - 1)) : 0.0;   // one direction: no staples
  void* work = nullptr;
  if ((st = scratch_alloc(&work, links->bytes, s, "lq_ape_smear workspace")) != LQ_OK) return st;
  const size_t db = links->bytes / 4;
  for (int mu = 0; mu < 4 && st == LQ_OK; ++mu)   // unsmeared directions pass through both buffers
    if (!((dirs_mask >> mu) & 1u))
      st = cuda_check(cudaMemcpyAsync((char*)work + mu * db, (const char*)links->ptr + mu * db, db,
                                      cudaMemcpyDeviceToDevice, s),
                      "lq_ape_smear pass-through copy");
  const dim3 grid((unsigned)(((g.V + 127) / 128) * nd));
  for (int k = 0; k < n_steps && st == LQ_OK; ++k) {
    const void* in = (k % 2 == 0) ? links->ptr : work;
    void* out = (k % 2 == 0) ? work : links->ptr;
    if (links->prec == LQ_F64)
      k_ape<double><<<grid, 128, 0, s>>>((const double2*)in, (double2*)out, g, 1.0 - alpha, coef, dirs_mask, nd, ad);
    else
      k_ape<float><<<grid, 128, 0, s>>>((const float2*)in, (float2*)out, g, (float)(1.0 - alpha), (float)coef,
                                        dirs_mask, nd, ad);
    st = launch_check("lq_ape_smear kernel");
  }
  if (st == LQ_OK && n_steps % 2 == 1)
    for (int mu = 0; mu < 4 && st == LQ_OK; ++mu)
      if ((dirs_mask >> mu) & 1u)
        st = cuda_check(cudaMemcpyAsync((char*)links->ptr + mu * db, (const char*)work + mu * db, db,
                                        cudaMemcpyDeviceToDevice, s),
                        "lq_ape_smear result copy");
  scratch_free(work, s);
  return st;
}
