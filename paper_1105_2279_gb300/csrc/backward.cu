// Stout force: gradient of a scalar through n stout steps (Morningstar &
// Peardon 2004, Sec. IV), seeded by the Wilson-action gradient or by a given
// gradient field, with per-step checkpoints and forward recomputation.
//
// Convention: G_U = dS/dRe U + i dS/dIm U, so dS = Re tr(G^dag dU).  One step
// U -> U' (per smeared link: C = rho S, Omega = C U^dag, Q, E = exp(iQ),
// U' = E U) maps G' = G_{U'} to G_U in two kernels:
//   k_bwd_link:   per smeared link, G_E = G' U^dag,
//                 M = tr(G_E^dag B1) Q + tr(G_E^dag B2) Q^2 + f1 G_E^dag + f2 (Q G_E^dag + G_E^dag Q)
//                 with B_i = sum_j b_ij Q^j, G_Omega = TA(i M^dag);
//                 writes G_U(local) = E^dag G' + G_Omega^dag C and K = rho G_Omega U
//                 (the gradient w.r.t. the bare staple sum S).
//   k_bwd_staple: per link, adds the six staple-insertion terms of K of the
//                 neighbouring links (the six-term sum of the stout force).
// The APE force (lq_ape_backward) runs the same recursion with its own link
// kernel: per smeared link V = (1 - alpha) U + c S, U' = P(V), so
//   k_ape_bwd_link: G_V from G' through the projection (su3_project.cuh),
//                   writes G_U(local) = (1 - alpha) G_V and K = c G_V,
// followed by the same k_bwd_staple.
#include <algorithm>
#include <vector>

#include "lq_internal.h"
#include "stout_core.cuh"
#include "su3_project.cuh"

namespace lq {

template <typename R> using V2 = typename vec2<R>::type;

// sum_ij conj(A_ij) B_ij = tr(A^dag B)
template <typename R> __device__ __forceinline__ cx<R> tr_dn(const M3<R>& a, const M3<R>& b) {
  cx<R> t = mkc<R>(0, 0);
#pragma unroll
  for (int i = 0; i < 9; ++i) t = cfma_cn(a.e[i], b.e[i], t);
  return t;
}

template <typename R>
__global__ void __launch_bounds__(128) k_bwd_link(const V2<R>* __restrict__ U, const V2<R>* __restrict__ Gp,
                                                  V2<R>* __restrict__ Gout, V2<R>* __restrict__ K, GeomArgs g, R rho,
                                                  unsigned dirs) {
  const long long V = g.V;
  const long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  const int mu = blockIdx.y;
  const long long off = (long long)mu * 9 * V + s;
  if (!((dirs >> mu) & 1u)) {  // not smeared: the gradient passes through
    st_m3<R>(Gout + off, V, ld_m3<R>(Gp + off, V));
    return;
  }
  int c[4];
  site_coords(g, s, c);
  const M3<R> C = m_rscale(staple_sum<R>(U, g, s, c, mu, dirs), rho);
  const M3<R> Umu = ld_m3<R>(U + off, V);
  const QH<R> q = q_from_omega(mul_nd(C, Umu));
  const CHDeriv d = ch_coefficients_deriv<sizeof(R) == 4 ? 1 : 2>(
      to_f64(q.d0), to_f64(q.d1), to_f64(q.d2), mkc(to_f64(q.o01.re), to_f64(q.o01.im)),
      mkc(to_f64(q.o02.re), to_f64(q.o02.im)), mkc(to_f64(q.o12.re), to_f64(q.o12.im)));
  const QH<R> q2 = q_square(q);
  const M3<R> Qf = qh_full(q), Q2f = qh_full(q2);
  const M3<R> Gpm = ld_m3<R>(Gp + off, V);
  const M3<R> GE = mul_nd(Gpm, Umu);  // G_E = G' U^dag
  // tr(G_E^dag Q^j), j = 0, 1, 2
  const cx<R> t0 = cconj(m_trace(GE));
  const cx<R> t1 = tr_dn(GE, Qf);
  const cx<R> t2 = tr_dn(GE, Q2f);
  cx<double> a1 = mkc(0.0, 0.0), a2 = mkc(0.0, 0.0);
  const cx<double> td[3] = {mkc(to_f64(t0.re), to_f64(t0.im)), mkc(to_f64(t1.re), to_f64(t1.im)),
                            mkc(to_f64(t2.re), to_f64(t2.im))};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    a1 = cfma(d.b1[j], td[j], a1);
    a2 = cfma(d.b2[j], td[j], a2);
  }
  const cx<R> f1 = mkc<R>(from_f64<R>(d.f[1].re), from_f64<R>(d.f[1].im));
  const cx<R> f2 = mkc<R>(from_f64<R>(d.f[2].re), from_f64<R>(d.f[2].im));
  const M3<R> H = m_adj(GE);  // G_E^dag
  // M = a1 Q + a2 Q^2 + f1 H + f2 (Q H + H Q)
  M3<R> M = m_add(mul_nn(Qf, H), mul_nn(H, Qf));
  M = m_scale(M, f2);
  m_addto(M, m_scale(H, f1));
  m_addto(M, m_scale(Qf, mkc<R>(from_f64<R>(a1.re), from_f64<R>(a1.im))));
  m_addto(M, m_scale(Q2f, mkc<R>(from_f64<R>(a2.re), from_f64<R>(a2.im))));
  // G_Omega = TA(i M^dag)
  const M3<R> GO = m_ta(m_scale(m_adj(M), mkc<R>(0, 1)));
  // E = exp(iQ) and the local gradient E^dag G' + G_Omega^dag C
  const M3<R> E = expiq_assemble(q, q2, mkc<R>(from_f64<R>(d.f[0].re), from_f64<R>(d.f[0].im)), f1, f2);
  M3<R> Gl = mul_dn(E, Gpm);
  mac_dn(Gl, GO, C);
  st_m3<R>(Gout + off, V, Gl);
  st_m3<R>(K + off, V, m_rscale(mul_nn(GO, Umu), rho));
}

// APE step, per smeared link: V recomputed exactly as in the forward kernel
// (staples and mixing in the field precision), the projection's gradient in FP64.
template <typename R>
__global__ void __launch_bounds__(128) k_ape_bwd_link(const V2<R>* __restrict__ U, const V2<R>* __restrict__ Gp,
                                                      V2<R>* __restrict__ Gout, V2<R>* __restrict__ K, GeomArgs g,
                                                      R keep, R coef, unsigned dirs) {
  const long long V = g.V;
  const long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  const int mu = blockIdx.y;
  const long long off = (long long)mu * 9 * V + s;
  if (!((dirs >> mu) & 1u)) {  // not smeared: the gradient passes through
    st_m3<R>(Gout + off, V, ld_m3<R>(Gp + off, V));
    return;
  }
  int c[4];
  site_coords(g, s, c);
  const M3<R> C = staple_sum<R>(U, g, s, c, mu, dirs);
  const M3<R> Umu = ld_m3<R>(U + off, V);
  const M3<R> Gpm = ld_m3<R>(Gp + off, V);
  M3<double> v, gp;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<R> e = mkc<R>(fmaR(coef, C.e[i].re, keep * Umu.e[i].re), fmaR(coef, C.e[i].im, keep * Umu.e[i].im));
    v.e[i] = mkc(to_f64(e.re), to_f64(e.im));
    gp.e[i] = mkc(to_f64(Gpm.e[i].re), to_f64(Gpm.e[i].im));
  }
  const M3<double> gv = project_su3_vjp_f64<sizeof(R) == 4 ? 1 : 2>(v, gp);
  M3<R> gl, kk;
  const double kd = (double)keep, cd = (double)coef;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    gl.e[i] = mkc<R>(from_f64<R>(kd * gv.e[i].re), from_f64<R>(kd * gv.e[i].im));
    kk.e[i] = mkc<R>(from_f64<R>(cd * gv.e[i].re), from_f64<R>(cd * gv.e[i].im));
  }
  st_m3<R>(Gout + off, V, gl);
  st_m3<R>(K + off, V, kk);
}

template <typename R>
__device__ __forceinline__ M3<R> ld(const V2<R>* __restrict__ F, long long V, int dir, int s) {
  return ld_m3<R>(F + (long long)dir * 9 * V + s, V);
}

// G_alpha(y) += sum_{mu in dirs, mu != alpha} [ K_mu(y) U_a(y+mu) U_mu(y+a)^dag
//                 + K_mu(y-mu)^dag U_a(y-mu) U_mu(y-mu+a) + U_mu(y) U_a(y+mu) K_mu(y+a)^dag
//                 + U_mu(y-mu)^dag U_a(y-mu) K_mu(y-mu+a)
//                 + U_mu(y-mu)^dag K_a(y-mu) U_mu(y-mu+a) + U_mu(y) K_a(y+mu) U_mu(y+a)^dag ]
// The four directions of a block of sites run in consecutive CTAs, so the
// neighbour links and K they share are read while still in L2.
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1) k_bwd_staple(const V2<R>* __restrict__ U, const V2<R>* __restrict__ K,
                                                    V2<R>* __restrict__ G, GeomArgs g, unsigned dirs) {
  const long long V = g.V;
  const long long sl = (long long)(blockIdx.x / 4) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  const int a = blockIdx.x % 4;
  if (!((dirs >> a) & 1u)) return;
  int c[4];
  site_coords(g, s, c);
  const int s_pa = nb_fwd(g, s, coord_of(c, a), a);
  M3<R> acc = ld<R>(G, V, a, s);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (mu == a || !((dirs >> mu) & 1u)) continue;
    const int s_pmu = nb_fwd(g, s, c[mu], mu);
    const int s_mmu = nb_bwd(g, s, c[mu], mu);
    const int s_mmu_pa = nb_bwd(g, s_pa, c[mu], mu);  // y - mu + a
    // the three terms through y+mu, with A = U_mu(y), B = U_a(y+mu):
    //   (K_mu(y) B + A K_a(y+mu)) U_mu(y+a)^dag + (A B) K_mu(y+a)^dag   (5 products, not 6)
    {
      const M3<R> A = ld<R>(U, V, mu, s), B = ld<R>(U, V, a, s_pmu);
      M3<R> T = mul_nn(ld<R>(K, V, mu, s), B);
      mac_nn(T, A, ld<R>(K, V, a, s_pmu));
      mac_nd(acc, T, ld<R>(U, V, mu, s_pa));
      mac_nd(acc, mul_nn(A, B), ld<R>(K, V, mu, s_pa));
    }
    // the three terms through y-mu, with A = U_mu(y-mu), B = U_a(y-mu):
    //   (K_mu(y-mu)^dag B + A^dag K_a(y-mu)) U_mu(y-mu+a) + (A^dag B) K_mu(y-mu+a)
    {
      const M3<R> A = ld<R>(U, V, mu, s_mmu), B = ld<R>(U, V, a, s_mmu);
      M3<R> T = mul_dn(ld<R>(K, V, mu, s_mmu), B);
      mac_dn(T, A, ld<R>(K, V, a, s_mmu));
      mac_nn(acc, T, ld<R>(U, V, mu, s_mmu_pa));
      mac_nn(acc, mul_dn(A, B), ld<R>(K, V, mu, s_mmu_pa));
    }
  }
  st_m3<R>(G + (long long)a * 9 * V + s, V, acc);
}

// Wilson-action gradient G_mu(x) = -(beta/3) * (sum over all nu != mu of the staples).
template <typename R>
__global__ void __launch_bounds__(128) k_wilson_grad(const V2<R>* __restrict__ U, V2<R>* __restrict__ G, GeomArgs g,
                                                     R mbeta3) {
  const long long V = g.V;
  const long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  const int mu = blockIdx.y;
  int c[4];
  site_coords(g, s, c);
  st_m3<R>(G + (long long)mu * 9 * V + s, V, m_rscale(staple_sum<R>(U, g, s, c, mu, 15u), mbeta3));
}

// F_mu(x) = TA(G_mu(x) U_mu(x)^dag)
template <typename R>
__global__ void k_force(const V2<R>* __restrict__ U, const V2<R>* __restrict__ G, V2<R>* __restrict__ F, long long V) {
  const long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const long long off = (long long)blockIdx.y * 9 * V + sl;
  st_m3<R>(F + off, V, m_ta(mul_nd(ld_m3<R>(G + off, V), ld_m3<R>(U + off, V))));
}

struct Bufs {
  std::vector<void*> own;
  cudaStream_t s;
  ~Bufs() {
    for (void* p : own) scratch_free(p, s);
  }
};

enum class Smearing { kStout, kApe, kHyp };

// w: rho (stout) or alpha (APE); a[3] = (a1, a2, a3) for HYP
struct SmearArgs {
  Smearing kind;
  double w;
  double a[3];
};

template <typename R>
static lq_status backward_impl(const SmearArgs& sa, const lq_field* thin, int n, unsigned dirs,
                               const lq_field* seed, double beta, lq_field* force, lq_field* grad_out, int every,
                               cudaStream_t s) {
  const Smearing kind = sa.kind;
  const double w = sa.w;
  const char* who = kind == Smearing::kStout ? "lq_stout_backward"
                                             : (kind == Smearing::kApe ? "lq_ape_backward" : "lq_hyp_backward");
  const GeomArgs g = geom_args(thin->geom);
  const long long V = g.V;
  const size_t fb = thin->bytes;
  Bufs b;
  b.s = s;
  auto alloc = [&](void** p) -> lq_status {
    lq_status st = scratch_alloc(p, fb, s, who);
    if (st == LQ_OK) b.own.push_back(*p);
    return st;
  };
  lq_status st;
  // checkpoints: ck[j] holds U^(j) for j % every == 0 (ck[0] is the thin field itself)
  std::vector<void*> ck(n + 1, nullptr);
  ck[0] = thin->ptr;
  void *w0, *w1, *Ga, *Gb, *Kb = nullptr;   // Kb: staple-sum gradient (stout and APE only)
  if ((st = alloc(&w0)) || (st = alloc(&w1)) || (st = alloc(&Ga)) || (st = alloc(&Gb))) return st;
  if (kind != Smearing::kHyp && (st = alloc(&Kb))) return st;
  for (int j = every; j < n; j += every)
    if ((st = alloc(&ck[j]))) return st;
  void* hyp_scratch = nullptr;   // decorated links and their gradients
  if (kind == Smearing::kHyp && n > 0) {
    if ((st = scratch_alloc(&hyp_scratch, kHypBwdPlanes * (fb / 4), s, who))) return st;
    b.own.push_back(hyp_scratch);
  }
  TuneChoice tc = stout_default_choice(thin->prec);
  // recomputed fields follow lq_stout_smear's default (FP32 links are re-projected)
  const int reproject = thin->prec == LQ_F32 ? 1 : 0;
  auto run_steps = [&](void* links, int steps) -> lq_status {
    if (kind == Smearing::kApe) return ape_run_steps(links, w1, thin->geom, thin->prec, fb, w, steps, dirs, s);
    if (kind == Smearing::kHyp)
      return hyp_run_steps(links, w1, hyp_scratch, thin->geom, thin->prec, fb, sa.a[0], sa.a[1], sa.a[2], steps, s);
    return stout_run_steps(links, w1, thin->geom, thin->prec, w, steps, dirs, reproject, tc, s);
  };
  int nd = 0;
  for (int mu = 0; mu < 4; ++mu) nd += (dirs >> mu) & 1u;
  const double ape_coef = nd > 1 ? w / (2.0 * (nd - 1)) : 0.0;   // as in lq_ape_smear
  // forward: U^(j) from the nearest stored checkpoint at or below j (stored
  // indices are multiples of `every` below n), into dst
  auto forward_to = [&](int j, void* dst) -> lq_status {
    int j0 = (j / every) * every;
    if (j0 >= n) j0 = ((n - 1) / every) * every;
    lq_status st2 = cuda_check(cudaMemcpyAsync(dst, ck[j0], fb, cudaMemcpyDeviceToDevice, s), who);
    if (st2 != LQ_OK) return st2;
    return run_steps(dst, j - j0);
  };
  for (int j = every; j < n; j += every) {  // ck[j] = `every` steps from ck[j - every]
    if ((st = cuda_check(cudaMemcpyAsync(ck[j], ck[j - every], fb, cudaMemcpyDeviceToDevice, s), who)))
      return st;
    if ((st = run_steps(ck[j], every))) return st;
  }
  // seed at U^(n)
  if (seed) {
    if ((st = cuda_check(cudaMemcpyAsync(Ga, seed->ptr, fb, cudaMemcpyDeviceToDevice, s), who)))
      return st;
  } else {
    void* Un = thin->ptr;
    if (n > 0) {
      if ((st = forward_to(n, w0))) return st;
      Un = w0;
    }
    dim3 grid((unsigned)((V + 127) / 128), 4);
    k_wilson_grad<R><<<grid, 128, 0, s>>>((const V2<R>*)Un, (V2<R>*)Ga, g, (R)(-beta / 3.0));
    if ((st = launch_check("k_wilson_grad"))) return st;
  }
  for (int j = n - 1; j >= 0; --j) {
    const void* Uj = ck[j];
    if (!Uj) {
      if ((st = forward_to(j, w0))) return st;
      Uj = w0;
    }
    if (kind == Smearing::kHyp) {
      if ((st = hyp_backward_step(Uj, Ga, Gb, hyp_scratch, thin->geom, thin->prec, fb, sa.a[0], sa.a[1], sa.a[2], s)))
        return st;
      std::swap(Ga, Gb);
      continue;
    }
    dim3 grid((unsigned)((V + 127) / 128), 4);
    if (kind == Smearing::kApe)
      k_ape_bwd_link<R><<<grid, 128, 0, s>>>((const V2<R>*)Uj, (const V2<R>*)Ga, (V2<R>*)Gb, (V2<R>*)Kb, g,
                                             (R)(1.0 - w), (R)ape_coef, dirs);
    else
      k_bwd_link<R><<<grid, 128, 0, s>>>((const V2<R>*)Uj, (const V2<R>*)Ga, (V2<R>*)Gb, (V2<R>*)Kb, g, (R)w, dirs);
    if ((st = launch_check("backward link kernel"))) return st;
    k_bwd_staple<R><<<grid.x * 4, 128, 0, s>>>((const V2<R>*)Uj, (const V2<R>*)Kb, (V2<R>*)Gb, g, dirs);
    if ((st = launch_check("k_bwd_staple"))) return st;
    std::swap(Ga, Gb);
  }
  if (force) {
    dim3 grid((unsigned)((V + 255) / 256), 4);
    k_force<R><<<grid, 256, 0, s>>>((const V2<R>*)thin->ptr, (const V2<R>*)Ga, (V2<R>*)force->ptr, V);
    if ((st = launch_check("k_force"))) return st;
  }
  if (grad_out)
    if ((st = cuda_check(cudaMemcpyAsync(grad_out->ptr, Ga, fb, cudaMemcpyDeviceToDevice, s), who)))
      return st;
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

// Argument checks shared by the two force entry points.
static lq_status check_backward(const char* who, const lq_field* thin, unsigned dirs_mask, int n_steps, double beta,
                                const lq_field* grad_seed, const lq_field* force_out, const lq_field* grad_out) {
  lq_status st = check_links(thin, who);
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, who)) != LQ_OK) return st;
  if (n_steps < 0 || !(beta == beta)) {
    set_error("%s: n_steps must be >= 0 and beta finite", who);
    return LQ_ERR_ARG;
  }
  if (!force_out && !grad_out) {
    set_error("%s: neither force_out nor grad_out given", who);
    return LQ_ERR_ARG;
  }
  const lq_field* outs[3] = {grad_seed, force_out, grad_out};
  for (const lq_field* f : outs) {
    if (!f) continue;
    if (f->kind != LQ_LINKS || f->prec != thin->prec || !same_geom(f->geom, thin->geom)) {
      set_error("%s: seed/force/grad fields must be LINKS of the thin field's geometry and precision", who);
      return LQ_ERR_GEOM;
    }
    if (f->ptr == thin->ptr) {
      set_error("%s: outputs must not alias the thin links", who);
      return LQ_ERR_ARG;
    }
  }
  return LQ_OK;
}

static int checkpoint_every(const lq_backward_opts* opts) {
  if (opts && opts->struct_size >= (int)sizeof(lq_backward_opts) && opts->checkpoint_every > 0)
    return opts->checkpoint_every;
  return 1;
}

extern "C" lq_status lq_stout_backward(const lq_field* thin, double rho, int n_steps, unsigned dirs_mask,
                                       const lq_field* grad_seed, double beta, lq_field* force_out, lq_field* grad_out,
                                       const lq_backward_opts* opts, void* stream) {
  clear_error();
  lq_status st = check_backward("lq_stout_backward", thin, dirs_mask, n_steps, beta, grad_seed, force_out, grad_out);
  if (st != LQ_OK) return st;
  if (!(rho >= 0.0) || rho > 1e6) {
    set_error("lq_stout_backward: rho must be finite >= 0");
    return LQ_ERR_ARG;
  }
  const int every = checkpoint_every(opts);
  cudaStream_t s = as_stream(stream);
  if (thin->prec == LQ_F64)
    return backward_impl<double>(SmearArgs{Smearing::kStout, rho, {0, 0, 0}}, thin, n_steps, dirs_mask, grad_seed,
                                 beta, force_out, grad_out, every, s);
  return backward_impl<float>(SmearArgs{Smearing::kStout, rho, {0, 0, 0}}, thin, n_steps, dirs_mask, grad_seed, beta,
                              force_out, grad_out, every, s);
}

extern "C" lq_status lq_ape_backward(const lq_field* thin, double alpha, int n_steps, unsigned dirs_mask,
                                     const lq_field* grad_seed, double beta, lq_field* force_out, lq_field* grad_out,
                                     const lq_backward_opts* opts, void* stream) {
  clear_error();
  lq_status st = check_backward("lq_ape_backward", thin, dirs_mask, n_steps, beta, grad_seed, force_out, grad_out);
  if (st != LQ_OK) return st;
  if (!(alpha == alpha) || alpha > 1e6 || alpha < -1e6) {
    set_error("lq_ape_backward: alpha must be finite");
    return LQ_ERR_ARG;
  }
  const int every = checkpoint_every(opts);
  cudaStream_t s = as_stream(stream);
  if (thin->prec == LQ_F64)
    return backward_impl<double>(SmearArgs{Smearing::kApe, alpha, {0, 0, 0}}, thin, n_steps, dirs_mask, grad_seed,
                                 beta, force_out, grad_out, every, s);
  return backward_impl<float>(SmearArgs{Smearing::kApe, alpha, {0, 0, 0}}, thin, n_steps, dirs_mask, grad_seed, beta,
                              force_out, grad_out, every, s);
}

extern "C" lq_status lq_hyp_backward(const lq_field* thin, double a1, double a2, double a3, int n_steps,
                                     const lq_field* grad_seed, double beta, lq_field* force_out, lq_field* grad_out,
                                     const lq_backward_opts* opts, void* stream) {
  clear_error();
  lq_status st = check_backward("lq_hyp_backward", thin, 15u, n_steps, beta, grad_seed, force_out, grad_out);
  if (st != LQ_OK) return st;
  const double as[3] = {a1, a2, a3};
  for (double a : as)
    if (!(a == a) || a > 1e6 || a < -1e6) {
      set_error("lq_hyp_backward: the weights must be finite");
      return LQ_ERR_ARG;
    }
  const int every = checkpoint_every(opts);
  cudaStream_t s = as_stream(stream);
  const SmearArgs sa{Smearing::kHyp, 0.0, {a1, a2, a3}};
  if (thin->prec == LQ_F64)
    return backward_impl<double>(sa, thin, n_steps, 15u, grad_seed, beta, force_out, grad_out, every, s);
  return backward_impl<float>(sa, thin, n_steps, 15u, grad_seed, beta, force_out, grad_out, every, s);
}
