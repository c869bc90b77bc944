// HYP smearing (A. Hasenfratz and F. Knechtli, Phys. Rev. D 64 (2001)
// 034504) of a 4D LINKS field: three nested APE-type levels whose staples stay
// inside the hypercubes attached to the link, each level projected to SU(3)
// (su3_project.cuh).  With S(A, B, mu, eta) the forward + backward staple of
// the direction pair (mu, eta) from transverse links A_eta and links B_mu along mu,
//   A_eta(x) B_mu(x+eta) A_eta(x+mu)^dag + A_eta(x-eta)^dag B_mu(x-eta) A_eta(x-eta+mu):
//   level 3  Vb[mu][eta] = P((1 - a3) U_mu + a3/2 S(U, U, mu, eta))              (12 fields)
//   level 2  Vt[mu][nu]  = P((1 - a2) U_mu + a2/4 sum_{rho not in {mu,nu}}
//                                  S(Vb[rho][sigma], Vb[mu][sigma], mu, rho))   (12 fields)
//            sigma the fourth direction, not in {mu, nu, rho}
//   level 1  U'_mu       = P((1 - a1) U_mu + a1/6 sum_{nu != mu} S(Vt[nu][mu], Vt[mu][nu], mu, nu))
// One kernel per level; the decorated links live in two scratch buffers of
// 12 colour-matrix fields in the field precision.  Mixing and staples run in
// the field precision, the projections in FP64.
#include "lq_internal.h"
#include "stout_core.cuh"
#include "su3_project.cuh"

namespace lq {

// index of the ordered pair (a, b), a != b, among the 12
__host__ __device__ constexpr int pair_index(int a, int b) { return 3 * a + (b < a ? b : b - 1); }

template <typename R>
__device__ __forceinline__ M3<R> ld_plane(const typename vec2<R>::type* __restrict__ F, long long V, int plane, int s) {
  return ld_m3<R>(F + (long long)plane * 9 * V + s, V);
}

// site of x +- one step along d
__device__ __forceinline__ int step(const GeomArgs& g, int s, const int c[4], int d, int sign) {
  return sign > 0 ? nb_fwd(g, s, coord_of(c, d), d) : nb_bwd(g, s, coord_of(c, d), d);
}

// acc += A_eta(x) B_mu(x+eta) A_eta(x+mu)^dag + A_eta(x-eta)^dag B_mu(x-eta) A_eta(x-eta+mu),
// A_eta in plane pa of F, B_mu in plane pb of F
template <typename R>
__device__ __forceinline__ void add_staples(M3<R>& acc, const typename vec2<R>::type* __restrict__ F, long long V,
                                            int pa, int pb, const GeomArgs& g, int s, const int c[4], int mu,
                                            int eta) {
  const int s_pe = step(g, s, c, eta, +1), s_pm = step(g, s, c, mu, +1), s_me = step(g, s, c, eta, -1);
  int cm[4] = {c[0], c[1], c[2], c[3]};
  cm[eta] = coord_of(c, eta) > 0 ? coord_of(c, eta) - 1 : g.L[eta] - 1;
  const int s_me_pm = step(g, s_me, cm, mu, +1);
  mac_nn(acc, ld_plane<R>(F, V, pa, s), mul_nd(ld_plane<R>(F, V, pb, s_pe), ld_plane<R>(F, V, pa, s_pm)));
  const M3<R> Am = ld_plane<R>(F, V, pa, s_me);
  mac_dn(acc, Am, mul_nn(ld_plane<R>(F, V, pb, s_me), ld_plane<R>(F, V, pa, s_me_pm)));
}

template <typename R>
__device__ __forceinline__ M3<R> mix_project(const M3<R>& U, const M3<R>& S, R keep, R coef) {
  M3<double> v;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<R> e = mkc<R>(fmaR(coef, S.e[i].re, keep * U.e[i].re), fmaR(coef, S.e[i].im, keep * U.e[i].im));
    v.e[i] = mkc(to_f64(e.re), to_f64(e.im));
  }
  const M3<double> P = project_su3_f64<sizeof(R) == 4 ? 1 : 2>(v);
  M3<R> out;
#pragma unroll
  for (int i = 0; i < 9; ++i) out.e[i] = mkc<R>(from_f64<R>(P.e[i].re), from_f64<R>(P.e[i].im));
  return out;
}

// the (mu, other) pair of a thread: the 12 pairs of a site block run in consecutive CTAs
__device__ __forceinline__ void block_pair(int* mu, int* other) {
  const int p = blockIdx.x % 12;
  *mu = p / 3;
  const int o = p % 3;
  *other = o < *mu ? o : o + 1;
}

// level 3: Vb[mu][eta], the link field U given as planes 0..3 (its own layout)
template <typename R>
__global__ void __launch_bounds__(128) k_hyp3(const typename vec2<R>::type* __restrict__ U,
                                              typename vec2<R>::type* __restrict__ Vb, GeomArgs g, R keep, R coef) {
  int mu, eta;
  block_pair(&mu, &eta);
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 12) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  M3<R> S;
  m_zero(S);
  add_staples<R>(S, U, V, eta, mu, g, s, c, mu, eta);
  st_m3<R>(Vb + (long long)pair_index(mu, eta) * 9 * V + s, V, mix_project<R>(ld_plane<R>(U, V, mu, s), S, keep, coef));
}

// level 2: Vt[mu][nu] from Vb
template <typename R>
__global__ void __launch_bounds__(128) k_hyp2(const typename vec2<R>::type* __restrict__ U,
                                              const typename vec2<R>::type* __restrict__ Vb,
                                              typename vec2<R>::type* __restrict__ Vt, GeomArgs g, R keep, R coef) {
  int mu, nu;
  block_pair(&mu, &nu);
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 12) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  M3<R> S;
  m_zero(S);
#pragma unroll 1
  for (int rho = 0; rho < 4; ++rho) {
    if (rho == mu || rho == nu) continue;
    const int sigma = 6 - mu - nu - rho;
    add_staples<R>(S, Vb, V, pair_index(rho, sigma), pair_index(mu, sigma), g, s, c, mu, rho);
  }
  st_m3<R>(Vt + (long long)pair_index(mu, nu) * 9 * V + s, V, mix_project<R>(ld_plane<R>(U, V, mu, s), S, keep, coef));
}

// level 1: U'_mu from Vt (transverse Vt[nu][mu], along mu Vt[mu][nu]): the
// pair planes differ per staple, so the two loads name their planes
template <typename R>
__global__ void __launch_bounds__(128) k_hyp1(const typename vec2<R>::type* __restrict__ U,
                                              const typename vec2<R>::type* __restrict__ Vt,
                                              typename vec2<R>::type* __restrict__ Uout, GeomArgs g, R keep, R coef) {
  const int mu = blockIdx.x % 4;
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 4) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  M3<R> S;
  m_zero(S);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    add_staples<R>(S, Vt, V, pair_index(nu, mu), pair_index(mu, nu), g, s, c, mu, nu);
  }
  st_m3<R>(Uout + (long long)mu * 9 * V + s, V, mix_project<R>(ld_plane<R>(U, V, mu, s), S, keep, coef));
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_hyp_smear(lq_field* links, double a1, double a2, double a3, int n_steps, void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_hyp_smear");
  if (st != LQ_OK) return st;
  const double as[3] = {a1, a2, a3};
  for (double a : as)
    if (!(a == a) || a > 1e6 || a < -1e6) {
      set_error("lq_hyp_smear: the weights must be finite");
      return LQ_ERR_ARG;
    }
  if (n_steps < 0) {
    set_error("lq_hyp_smear: n_steps must be >= 0");
    return LQ_ERR_ARG;
  }
  if (n_steps == 0) return LQ_OK;
  cudaStream_t s = as_stream(stream);
  const GeomArgs g = geom_args(links->geom);
  void *vb = nullptr, *vt = nullptr, *work = nullptr;
  const size_t plane_bytes = links->bytes / 4;
  if ((st = scratch_alloc(&vb, 12 * plane_bytes, s, "lq_hyp_smear level-3 links")) != LQ_OK) return st;
  if ((st = scratch_alloc(&vt, 12 * plane_bytes, s, "lq_hyp_smear level-2 links")) != LQ_OK) {
    scratch_free(vb, s);
    return st;
  }
  if ((st = scratch_alloc(&work, links->bytes, s, "lq_hyp_smear workspace")) != LQ_OK) {
    scratch_free(vb, s);
    scratch_free(vt, s);
    return st;
  }
  const unsigned blocks = (unsigned)((g.V + 127) / 128);
  for (int k = 0; k < n_steps && st == LQ_OK; ++k) {
    const void* in = (k % 2 == 0) ? links->ptr : work;
    void* out = (k % 2 == 0) ? work : links->ptr;
    if (links->prec == LQ_F64) {
      k_hyp3<double><<<blocks * 12, 128, 0, s>>>((const double2*)in, (double2*)vb, g, 1.0 - a3, a3 / 2.0);
      k_hyp2<double><<<blocks * 12, 128, 0, s>>>((const double2*)in, (const double2*)vb, (double2*)vt, g, 1.0 - a2,
                                                 a2 / 4.0);
      k_hyp1<double><<<blocks * 4, 128, 0, s>>>((const double2*)in, (const double2*)vt, (double2*)out, g, 1.0 - a1,
                                                a1 / 6.0);
    } else {
      k_hyp3<float><<<blocks * 12, 128, 0, s>>>((const float2*)in, (float2*)vb, g, (float)(1.0 - a3), (float)(a3 / 2.0));
      k_hyp2<float><<<blocks * 12, 128, 0, s>>>((const float2*)in, (const float2*)vb, (float2*)vt, g,
                                                (float)(1.0 - a2), (float)(a2 / 4.0));
      k_hyp1<float><<<blocks * 4, 128, 0, s>>>((const float2*)in, (const float2*)vt, (float2*)out, g,
                                               (float)(1.0 - a1), (float)(a1 / 6.0));
    }
    st = launch_check("lq_hyp_smear kernels");
  }
  if (st == LQ_OK && n_steps % 2 == 1)
    st = cuda_check(cudaMemcpyAsync(links->ptr, work, links->bytes, cudaMemcpyDeviceToDevice, s), "lq_hyp_smear copy");
  scratch_free(vb, s);
  scratch_free(vt, s);
  scratch_free(work, s);
  return st;
}
