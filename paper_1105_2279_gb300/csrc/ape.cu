// APE link smearing (M. Albanese et al., Phys. Lett. B 192 (1987) 163), an
// adjacent smearing on the same staple sum as the stout step:
//   V_mu(x) = (1 - alpha) U_mu(x) + alpha / (2 (d - 1)) * C_mu(x),   d = |dirs|,
//   U'_mu(x) = P(V_mu(x)),
// C the staple sum of the stout step (without rho) and P the projection to
// SU(3) by the unitary polar factor with the determinant phase removed:
//   W = V (V^dag V)^(-1/2),   P(V) = W exp(-i arg(det W) / 3),   arg in (-pi, pi].
// The mixing runs in the field precision, P always in FP64.
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
  const double sp = sqrt(p);
  const double r = sp > 0.0 ? fmin(fabs(q) / (p * sp), 1.0) : 0.0;
  const double y = cos_third_acos<2>(r);
  const double z = sqrt(fmax(1.0 - y * y, 0.0));
  const double sg = q < 0.0 ? -1.0 : 1.0;
  const double l1 = m + sg * 2.0 * sp * y;
  const double l2 = m + sg * sp * (-y + 1.7320508075688772 * z);
  const double l3 = m + sg * sp * (-y - 1.7320508075688772 * z);
  const double s1 = sqrt(l1), s2 = sqrt(l2), s3 = sqrt(l3);
  const double d1 = 1.0 / s1;
  const double d12 = -1.0 / (s1 * s2 * (s1 + s2));
  const double d123 = (s1 + s2 + s3) / (s1 * s2 * s3 * (s1 + s2) * (s2 + s3) * (s1 + s3));
  // X = d1 + d12 (A - l1) + d123 (A - l1)(A - l2) = c0 + c1 A + c2 A^2
  const double c2 = d123, c1 = d12 - d123 * (l1 + l2), c0 = d1 - d12 * l1 + d123 * l1 * l2;
  M3<double> A;
  A.e[0] = mkc(a00, 0.0);
  A.e[4] = mkc(a11, 0.0);
  A.e[8] = mkc(a22, 0.0);
  A.e[1] = a01;
  A.e[2] = a02;
  A.e[5] = a12;
  A.e[3] = cconj(a01);
  A.e[6] = cconj(a02);
  A.e[7] = cconj(a12);
  const M3<double> A2 = mul_nn(A, A);
  M3<double> X;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    X.e[i] = mkc(fma(c2, A2.e[i].re, c1 * A.e[i].re), fma(c2, A2.e[i].im, c1 * A.e[i].im));
  X.e[0].re += c0;
  X.e[4].re += c0;
  X.e[8].re += c0;
  M3<double> W = mul_nn(v, X);
  // det V, then exp(-i arg(det V) / 3)
  const cx<double> m0 = csub(cmul(v.e[4], v.e[8]), cmul(v.e[5], v.e[7]));
  const cx<double> m1 = csub(cmul(v.e[3], v.e[8]), cmul(v.e[5], v.e[6]));
  const cx<double> m2 = csub(cmul(v.e[3], v.e[7]), cmul(v.e[4], v.e[6]));
  const cx<double> det = cadd(csub(cmul(v.e[0], m0), cmul(v.e[1], m1)), cmul(v.e[2], m2));
  double sn, cs;
  sincos_red(atan2(det.im, det.re) * (1.0 / 3.0), &sn, &cs);
  const cx<double> ph = mkc(cs, -sn);
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
  const M3<double> P = project_su3_f64(v);
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
