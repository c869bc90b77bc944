// APE link smearing (M. Albanese et al., Phys. Lett. B 192 (1987) 163), an
// adjacent smearing on the same staple sum as the stout step:
//   V_mu(x) = (1 - alpha) U_mu(x) + alpha / (2 (d - 1)) * C_mu(x),   d = |dirs|,
//   U'_mu(x) = P(V_mu(x)),
// C the staple sum of the stout step (without rho) and P the projection to
// SU(3) by the unitary polar factor with the determinant phase removed:
//   W = V (V^dag V)^(-1/2),   P(V) = W exp(-i arg(det W) / 3),   arg in (-pi, pi].
// The mixing runs in the field precision, P (su3_project.cuh) always in FP64.
#include "lq_internal.h"
#include "stout_core.cuh"
#include "su3_project.cuh"

namespace lq {

struct ApeDirs {
  int mu[4];
};

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

namespace lq {

static ApeDirs ape_dirs(unsigned dirs_mask, int* nd_out) {
  ApeDirs ad;
  int nd = 0;
  for (int mu = 0; mu < 4; ++mu)
    if ((dirs_mask >> mu) & 1u) ad.mu[nd++] = mu;
  for (int j = nd; j < 4; ++j) ad.mu[j] = 0;
  *nd_out = nd;
  return ad;
}

lq_status ape_step(const void* in, void* out, const lq_geom& geom, int prec, double alpha, unsigned dirs_mask,
                   cudaStream_t s) {
  const GeomArgs g = geom_args(geom);
  int nd = 0;
  const ApeDirs ad = ape_dirs(dirs_mask, &nd);
  const double coef = nd > 1 ? alpha / (2.0 * (nd - 1)) : 0.0;   // one direction: no staples
  const dim3 grid((unsigned)(((g.V + 127) / 128) * nd));
  if (prec == LQ_F64)
    k_ape<double><<<grid, 128, 0, s>>>((const double2*)in, (double2*)out, g, 1.0 - alpha, coef, dirs_mask, nd, ad);
  else
    k_ape<float><<<grid, 128, 0, s>>>((const float2*)in, (float2*)out, g, (float)(1.0 - alpha), (float)coef,
                                      dirs_mask, nd, ad);
  return launch_check("lq_ape_smear kernel");
}

lq_status ape_run_steps(void* links, void* work, const lq_geom& geom, int prec, size_t bytes, double alpha,
                        int n_steps, unsigned dirs_mask, cudaStream_t s) {
  if (n_steps == 0) return LQ_OK;
  const size_t db = bytes / 4;
  lq_status st = LQ_OK;
  for (int mu = 0; mu < 4 && st == LQ_OK; ++mu)   // unsmeared directions pass through both buffers
    if (!((dirs_mask >> mu) & 1u))
      st = cuda_check(cudaMemcpyAsync((char*)work + mu * db, (const char*)links + mu * db, db,
                                      cudaMemcpyDeviceToDevice, s),
                      "lq_ape_smear pass-through copy");
  for (int k = 0; k < n_steps && st == LQ_OK; ++k) {
    const void* in = (k % 2 == 0) ? links : work;
    void* out = (k % 2 == 0) ? work : links;
    st = ape_step(in, out, geom, prec, alpha, dirs_mask, s);
  }
  if (st == LQ_OK && n_steps % 2 == 1)
    for (int mu = 0; mu < 4 && st == LQ_OK; ++mu)
      if ((dirs_mask >> mu) & 1u)
        st = cuda_check(cudaMemcpyAsync((char*)links + mu * db, (const char*)work + mu * db, db,
                                        cudaMemcpyDeviceToDevice, s),
                        "lq_ape_smear result copy");
  return st;
}

}  // namespace lq

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
  void* work = nullptr;
  if ((st = scratch_alloc(&work, links->bytes, s, "lq_ape_smear workspace")) != LQ_OK) return st;
  st = ape_run_steps(links->ptr, work, links->geom, links->prec, links->bytes, alpha, n_steps, dirs_mask, s);
  scratch_free(work, s);
  return st;
}
