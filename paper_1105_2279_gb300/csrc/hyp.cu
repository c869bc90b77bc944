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
//
// The force (lq_hyp_backward) runs the levels backwards per step: the
// gradient at each level's sum V from the projection's gradient
// (su3_project.cuh), then gather kernels that collect, for every decorated
// (or thin) link, the staple terms of the next level that read it.  With
// K = c G_V the staple gradient of S(A, B, mu, eta), a link T receives
//   as A (transverse):  K(y) T(y+mu) B(y+eta)^dag + K(y-mu)^dag T(y-mu) B(y-mu+eta)
//                       + B(y) T(y+mu) K(y+eta)^dag + B(y-mu)^dag T(y-mu) K(y-mu+eta)
//   as B (along mu):    A(y-eta)^dag K(y-eta) A(y-eta+mu) + A(y) K(y+eta) A(y+mu)^dag.
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

// ---- force --------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ M3<double> mix_f64(const M3<R>& U, const M3<R>& S, R keep, R coef) {
  M3<double> v;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<R> e = mkc<R>(fmaR(coef, S.e[i].re, keep * U.e[i].re), fmaR(coef, S.e[i].im, keep * U.e[i].im));
    v.e[i] = mkc(to_f64(e.re), to_f64(e.im));
  }
  return v;
}

// G_V = P'(V)^* G_P in FP64, G_P given in the field precision; the result rounded to it
template <typename R>
__device__ __forceinline__ M3<R> proj_grad(const M3<double>& v, const M3<R>& gp) {
  M3<double> g;
#pragma unroll
  for (int i = 0; i < 9; ++i) g.e[i] = mkc(to_f64(gp.e[i].re), to_f64(gp.e[i].im));
  const M3<double> gv = project_su3_vjp_f64<sizeof(R) == 4 ? 1 : 2>(v, g);
  M3<R> out;
#pragma unroll
  for (int i = 0; i < 9; ++i) out.e[i] = mkc<R>(from_f64<R>(gv.e[i].re), from_f64<R>(gv.e[i].im));
  return out;
}

// T (plane pt of TF) as the transverse field A of S(A, B, mu, eta), B in plane
// pb of BF, K in plane pk of KF: the four terms of the header
template <typename R>
__device__ __forceinline__ void gather_a(M3<R>& acc, const typename vec2<R>::type* __restrict__ TF, int pt,
                                         const typename vec2<R>::type* __restrict__ BF, int pb,
                                         const typename vec2<R>::type* __restrict__ KF, int pk, long long V,
                                         const GeomArgs& g, int s, const int c[4], int mu, int eta) {
  const int s_pm = step(g, s, c, mu, +1), s_mm = step(g, s, c, mu, -1), s_pe = step(g, s, c, eta, +1);
  const int s_mm_pe = nb_fwd(g, s_mm, coord_of(c, eta), eta);   // y - mu + eta (mu != eta)
  const M3<R> Tp = ld_plane<R>(TF, V, pt, s_pm);
  mac_nd(acc, mul_nn(ld_plane<R>(KF, V, pk, s), Tp), ld_plane<R>(BF, V, pb, s_pe));
  mac_nd(acc, mul_nn(ld_plane<R>(BF, V, pb, s), Tp), ld_plane<R>(KF, V, pk, s_pe));
  const M3<R> Tm = ld_plane<R>(TF, V, pt, s_mm);
  mac_nn(acc, mul_dn(ld_plane<R>(KF, V, pk, s_mm), Tm), ld_plane<R>(BF, V, pb, s_mm_pe));
  mac_nn(acc, mul_dn(ld_plane<R>(BF, V, pb, s_mm), Tm), ld_plane<R>(KF, V, pk, s_mm_pe));
}

// T as the field B along mu of S(A, T, mu, eta), A in plane pa of AF: the two terms
template <typename R>
__device__ __forceinline__ void gather_b(M3<R>& acc, const typename vec2<R>::type* __restrict__ AF, int pa,
                                         const typename vec2<R>::type* __restrict__ KF, int pk, long long V,
                                         const GeomArgs& g, int s, const int c[4], int mu, int eta) {
  const int s_me = step(g, s, c, eta, -1), s_pe = step(g, s, c, eta, +1), s_pm = step(g, s, c, mu, +1);
  const int s_me_pm = nb_fwd(g, s_me, coord_of(c, mu), mu);     // y - eta + mu (mu != eta)
  mac_nn(acc, mul_dn(ld_plane<R>(AF, V, pa, s_me), ld_plane<R>(KF, V, pk, s_me)), ld_plane<R>(AF, V, pa, s_me_pm));
  mac_nd(acc, mul_nn(ld_plane<R>(AF, V, pa, s), ld_plane<R>(KF, V, pk, s_pe)), ld_plane<R>(AF, V, pa, s_pm));
}

template <typename R>
__device__ __forceinline__ void st_plane(typename vec2<R>::type* __restrict__ F, long long V, int plane, int s,
                                         const M3<R>& m) {
  st_m3<R>(F + (long long)plane * 9 * V + s, V, m);
}

// level 1: GV1[mu] = gradient at V1[mu] from Gp[mu]
template <typename R>
__global__ void __launch_bounds__(128) k_hyp1_bwd(const typename vec2<R>::type* __restrict__ U,
                                                  const typename vec2<R>::type* __restrict__ Vt,
                                                  const typename vec2<R>::type* __restrict__ Gp,
                                                  typename vec2<R>::type* __restrict__ GV1, GeomArgs g, R keep,
                                                  R coef) {
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
  st_plane<R>(GV1, V, mu, s,
              proj_grad<R>(mix_f64<R>(ld_plane<R>(U, V, mu, s), S, keep, coef), ld_plane<R>(Gp, V, mu, s)));
}

// G_Vt[m][n] = coef * (Vt[m][n] as A in link n's staple with eta = m, K = GV1[n];
//                      as B in link m's staple with eta = n, K = GV1[m])
template <typename R>
__global__ void __launch_bounds__(128) k_hyp_gather1(const typename vec2<R>::type* __restrict__ Vt,
                                                     const typename vec2<R>::type* __restrict__ GV1,
                                                     typename vec2<R>::type* __restrict__ GT, GeomArgs g, R coef) {
  int m, n;
  block_pair(&m, &n);
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 12) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  M3<R> acc;
  m_zero(acc);
  gather_a<R>(acc, Vt, pair_index(m, n), Vt, pair_index(n, m), GV1, n, V, g, s, c, n, m);
  gather_b<R>(acc, Vt, pair_index(n, m), GV1, m, V, g, s, c, m, n);
  st_plane<R>(GT, V, pair_index(m, n), s, m_rscale(acc, coef));
}

// level 2: GV2[mu][nu] = gradient at V2[mu][nu] from G_Vt[mu][nu]
template <typename R>
__global__ void __launch_bounds__(128) k_hyp2_bwd(const typename vec2<R>::type* __restrict__ U,
                                                  const typename vec2<R>::type* __restrict__ Vb,
                                                  const typename vec2<R>::type* __restrict__ GT,
                                                  typename vec2<R>::type* __restrict__ GV2, GeomArgs g, R keep,
                                                  R coef) {
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
  const int p = pair_index(mu, nu);
  st_plane<R>(GV2, V, p, s, proj_grad<R>(mix_f64<R>(ld_plane<R>(U, V, mu, s), S, keep, coef), ld_plane<R>(GT, V, p, s)));
}

// G_Vb[r][s] = coef * (Vb[r][s] as A in the staples of V2[p][q] and V2[q][p] with eta = r
//                      (B = Vb[p][s], Vb[q][s]); as B in those of V2[r][p] (eta = q, A = Vb[q][s])
//                      and V2[r][q] (eta = p, A = Vb[p][s])), {p, q} the two other directions
template <typename R>
__global__ void __launch_bounds__(128) k_hyp_gather2(const typename vec2<R>::type* __restrict__ Vb,
                                                     const typename vec2<R>::type* __restrict__ GV2,
                                                     typename vec2<R>::type* __restrict__ GT, GeomArgs g, R coef) {
  int r, sg;
  block_pair(&r, &sg);
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 12) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  int p = 0;
  while (p == r || p == sg) ++p;
  const int q = 6 - r - sg - p;
  const int t = pair_index(r, sg);
  M3<R> acc;
  m_zero(acc);
  gather_a<R>(acc, Vb, t, Vb, pair_index(p, sg), GV2, pair_index(p, q), V, g, s, c, p, r);
  gather_a<R>(acc, Vb, t, Vb, pair_index(q, sg), GV2, pair_index(q, p), V, g, s, c, q, r);
  gather_b<R>(acc, Vb, pair_index(q, sg), GV2, pair_index(r, p), V, g, s, c, r, q);
  gather_b<R>(acc, Vb, pair_index(p, sg), GV2, pair_index(r, q), V, g, s, c, r, p);
  st_plane<R>(GT, V, t, s, m_rscale(acc, coef));
}

// level 3: GV3[mu][eta] = gradient at V3[mu][eta] from G_Vb[mu][eta]
template <typename R>
__global__ void __launch_bounds__(128) k_hyp3_bwd(const typename vec2<R>::type* __restrict__ U,
                                                  const typename vec2<R>::type* __restrict__ GT,
                                                  typename vec2<R>::type* __restrict__ GV3, GeomArgs g, R keep,
                                                  R coef) {
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
  const int p = pair_index(mu, eta);
  st_plane<R>(GV3, V, p, s, proj_grad<R>(mix_f64<R>(ld_plane<R>(U, V, mu, s), S, keep, coef), ld_plane<R>(GT, V, p, s)));
}

// G_U[a] = k1 GV1[a] + k2 sum_nu GV2[a][nu] + k3 sum_eta GV3[a][eta]
//          + coef (U_a as A in the staples of V3[mu][a], B = U_mu; as B in those of V3[a][eta], A = U_eta)
template <typename R>
__global__ void __launch_bounds__(128) k_hyp_gather3(const typename vec2<R>::type* __restrict__ U,
                                                     const typename vec2<R>::type* __restrict__ GV1,
                                                     const typename vec2<R>::type* __restrict__ GV2,
                                                     const typename vec2<R>::type* __restrict__ GV3,
                                                     typename vec2<R>::type* __restrict__ Gout, GeomArgs g, R k1, R k2,
                                                     R k3, R coef) {
  const int a = blockIdx.x % 4;
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 4) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  M3<R> st, loc = m_rscale(ld_plane<R>(GV1, V, a, s), k1);
  m_zero(st);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    if (mu == a) continue;
    gather_a<R>(st, U, a, U, mu, GV3, pair_index(mu, a), V, g, s, c, mu, a);
    gather_b<R>(st, U, mu, GV3, pair_index(a, mu), V, g, s, c, a, mu);
    const M3<R> g2 = ld_plane<R>(GV2, V, pair_index(a, mu), s), g3 = ld_plane<R>(GV3, V, pair_index(a, mu), s);
#pragma unroll
    for (int i = 0; i < 9; ++i)
      loc.e[i] = mkc<R>(fmaR(k3, g3.e[i].re, fmaR(k2, g2.e[i].re, loc.e[i].re)),
                        fmaR(k3, g3.e[i].im, fmaR(k2, g2.e[i].im, loc.e[i].im)));
  }
#pragma unroll
  for (int i = 0; i < 9; ++i)
    loc.e[i] = mkc<R>(fmaR(coef, st.e[i].re, loc.e[i].re), fmaR(coef, st.e[i].im, loc.e[i].im));
  st_plane<R>(Gout, V, a, s, loc);
}

template <typename R>
static void launch_forward_levels(const void* in, void* vb, void* vt, void* out, const GeomArgs& g, double a1,
                                  double a2, double a3, unsigned blocks, cudaStream_t s) {
  using T2 = typename vec2<R>::type;
  k_hyp3<R><<<blocks * 12, 128, 0, s>>>((const T2*)in, (T2*)vb, g, (R)(1.0 - a3), (R)(a3 / 2.0));
  k_hyp2<R><<<blocks * 12, 128, 0, s>>>((const T2*)in, (const T2*)vb, (T2*)vt, g, (R)(1.0 - a2), (R)(a2 / 4.0));
  if (out) k_hyp1<R><<<blocks * 4, 128, 0, s>>>((const T2*)in, (const T2*)vt, (T2*)out, g, (R)(1.0 - a1), (R)(a1 / 6.0));
}

lq_status hyp_run_steps(void* links, void* work, void* scratch, const lq_geom& geom, int prec, size_t bytes,
                        double a1, double a2, double a3, int n_steps, cudaStream_t s) {
  const GeomArgs g = geom_args(geom);
  const size_t plane_bytes = bytes / 4;
  void* vb = scratch;
  void* vt = (char*)scratch + 12 * plane_bytes;
  const unsigned blocks = (unsigned)((g.V + 127) / 128);
  lq_status st = LQ_OK;
  for (int k = 0; k < n_steps && st == LQ_OK; ++k) {
    const void* in = (k % 2 == 0) ? links : work;
    void* out = (k % 2 == 0) ? work : links;
    if (prec == LQ_F64) launch_forward_levels<double>(in, vb, vt, out, g, a1, a2, a3, blocks, s);
    else launch_forward_levels<float>(in, vb, vt, out, g, a1, a2, a3, blocks, s);
    st = launch_check("lq_hyp_smear kernels");
  }
  if (st == LQ_OK && n_steps % 2 == 1)
    st = cuda_check(cudaMemcpyAsync(links, work, bytes, cudaMemcpyDeviceToDevice, s), "lq_hyp_smear copy");
  return st;
}

template <typename R>
static lq_status hyp_backward_step_t(const void* Uk, const void* Gp, void* Gout, void* scratch, const GeomArgs& g,
                                     size_t plane_bytes, double a1, double a2, double a3, cudaStream_t s) {
  using T2 = typename vec2<R>::type;
  char* b = (char*)scratch;
  T2* vb = (T2*)b;
  T2* vt = (T2*)(b + 12 * plane_bytes);
  T2* gv1 = (T2*)(b + 24 * plane_bytes);
  T2* gv2 = (T2*)(b + 28 * plane_bytes);
  T2* gv3 = (T2*)(b + 40 * plane_bytes);
  T2* gt = (T2*)(b + 52 * plane_bytes);
  const T2* U = (const T2*)Uk;
  const unsigned blocks = (unsigned)((g.V + 127) / 128);
  launch_forward_levels<R>(Uk, vb, vt, nullptr, g, a1, a2, a3, blocks, s);
  k_hyp1_bwd<R><<<blocks * 4, 128, 0, s>>>(U, vt, (const T2*)Gp, gv1, g, (R)(1.0 - a1), (R)(a1 / 6.0));
  k_hyp_gather1<R><<<blocks * 12, 128, 0, s>>>(vt, gv1, gt, g, (R)(a1 / 6.0));
  k_hyp2_bwd<R><<<blocks * 12, 128, 0, s>>>(U, vb, gt, gv2, g, (R)(1.0 - a2), (R)(a2 / 4.0));
  k_hyp_gather2<R><<<blocks * 12, 128, 0, s>>>(vb, gv2, gt, g, (R)(a2 / 4.0));
  k_hyp3_bwd<R><<<blocks * 12, 128, 0, s>>>(U, gt, gv3, g, (R)(1.0 - a3), (R)(a3 / 2.0));
  k_hyp_gather3<R><<<blocks * 4, 128, 0, s>>>(U, gv1, gv2, gv3, (T2*)Gout, g, (R)(1.0 - a1), (R)(1.0 - a2),
                                              (R)(1.0 - a3), (R)(a3 / 2.0));
  return launch_check("lq_hyp_backward kernels");
}

lq_status hyp_backward_step(const void* Uk, const void* Gp, void* Gout, void* scratch, const lq_geom& geom, int prec,
                            size_t bytes, double a1, double a2, double a3, cudaStream_t s) {
  const GeomArgs g = geom_args(geom);
  if (prec == LQ_F64) return hyp_backward_step_t<double>(Uk, Gp, Gout, scratch, g, bytes / 4, a1, a2, a3, s);
  return hyp_backward_step_t<float>(Uk, Gp, Gout, scratch, g, bytes / 4, a1, a2, a3, s);
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
  void *scratch = nullptr, *work = nullptr;
  const size_t plane_bytes = links->bytes / 4;
  if ((st = scratch_alloc(&scratch, 24 * plane_bytes, s, "lq_hyp_smear decorated links")) != LQ_OK) return st;
  if ((st = scratch_alloc(&work, links->bytes, s, "lq_hyp_smear workspace")) != LQ_OK) {
    scratch_free(scratch, s);
    return st;
  }
  st = hyp_run_steps(links->ptr, work, scratch, links->geom, links->prec, links->bytes, a1, a2, a3, n_steps, s);
  scratch_free(scratch, s);
  scratch_free(work, s);
  return st;
}
