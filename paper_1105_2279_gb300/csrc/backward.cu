// Stout force: gradient of a scalar through n stout steps (Morningstar &
// Peardon 2004, Sec. IV), seeded by the Wilson-action gradient or by a given
// gradient field, with per-step checkpoints and forward recomputation.
//
// Convention: G_U = dS/dRe U + i dS/dIm U, so dS = Re tr(G^dag dU).  One step
// U -> U' (per smeared link: C = rho S, Omega = C U^dag, Q, E = exp(iQ),
// U' = E U) maps G' = G_{U'} to G_U in two stages:
//   link stage:   per smeared link, G_E = G' U^dag,
//                 M = tr(G_E^dag B1) Q + tr(G_E^dag B2) Q^2 + f1 G_E^dag + f2 (Q G_E^dag + G_E^dag Q)
//                 with B_i = sum_j b_ij Q^j, G_Omega = TA(i M^dag);
//                 G_U(local) = E^dag G' + G_Omega^dag C and K = rho G_Omega U
//                 (the gradient w.r.t. the bare staple sum S).
//   gather stage: per link, G_U = G_U(local) + the six staple-insertion terms
//                 of K of the neighbouring links (the six-term sum of the stout force).
// The gather of step j needs K of step j at neighbouring sites, so it cannot
// share a launch with the link stage of step j; but the link stage of step
// j-1 needs G at U^(j) only at its own link, which the gather of step j has
// just formed in registers.  One kernel per step therefore runs the gather of
// step j followed by the link stage of step j-1 on the same link: the FP32
// gather's loads and products interleave with the FP64 coefficient work of
// other warps, and G at U^(j) never goes through HBM.  The first kernel forms
// the seed (the Wilson-action gradient at U^(n), or a given field) in place of
// the gather, the last one writes the gradient and the force at the thin links
// in place of the link stage.
// The APE force (lq_ape_backward) runs the same recursion with its own link
// stage: per smeared link V = (1 - alpha) U + c S, U' = P(V), so
//   G_V from G' through the projection (su3_project.cuh),
//   G_U(local) = (1 - alpha) G_V and K = c G_V.
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
__device__ __forceinline__ M3<R> ld(const V2<R>* __restrict__ F, long long V, int dir, int s) {
  return ld_m3<R>(F + (long long)dir * 9 * V + s, V);
}

// Link stage of a stout step for the smeared link (s, mu), in two parts: the
// prefix recomputes the step's staple sum, Q and the FP64 coefficients with
// their derivatives (independent of the incoming gradient), the rest takes
// G' = the gradient at U'_mu(x) and returns G_U(local) in gl and K in kk.
template <typename R> struct StoutLinkPre {
  M3<R> C;
  QH<R> q;
  CHDeriv d;
};

template <typename R>
__device__ __forceinline__ void stout_link_pre(const V2<R>* __restrict__ U, const GeomArgs& g, int s, const int c[4],
                                               int mu, unsigned dirs, R rho, StoutLinkPre<R>& p) {
  p.C = m_rscale(staple_sum<R, true>(U, g, s, c, mu, dirs), rho);
  const QH<R> q = q_from_omega(mul_nd(p.C, ld<R>(U, g.V, mu, s)));
  p.q = q;
  p.d = ch_coefficients_deriv<sizeof(R) == 4 ? 1 : 2>(
      to_f64(q.d0), to_f64(q.d1), to_f64(q.d2), mkc(to_f64(q.o01.re), to_f64(q.o01.im)),
      mkc(to_f64(q.o02.re), to_f64(q.o02.im)), mkc(to_f64(q.o12.re), to_f64(q.o12.im)));
}

template <typename R>
__device__ __forceinline__ void stout_link_rest(const V2<R>* __restrict__ U, const GeomArgs& g, int s, int mu, R rho,
                                                const StoutLinkPre<R>& p, const M3<R>& Gpm, M3<R>& gl, M3<R>& kk) {
  const QH<R>& q = p.q;
  const CHDeriv& d = p.d;
  const M3<R> Umu = ld<R>(U, g.V, mu, s);
  const QH<R> q2 = q_square(q);
  const M3<R> Qf = qh_full(q), Q2f = qh_full(q2);
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
  gl = mul_dn(E, Gpm);
  mac_dn(gl, GO, p.C);
  kk = m_rscale(mul_nn(GO, Umu), rho);
}

// Link stage of an APE step: V recomputed exactly as in the forward kernel
// (staples and mixing in the field precision), the projection's gradient in FP64.
template <typename R>
__device__ __forceinline__ void ape_link_grad(const V2<R>* __restrict__ U, const GeomArgs& g, int s, const int c[4],
                                              int mu, unsigned dirs, R keep, R coef, const M3<R>& Gpm, M3<R>& gl,
                                              M3<R>& kk) {
  const long long V = g.V;
  const M3<R> C = staple_sum<R, true>(U, g, s, c, mu, dirs);
  const M3<R> Umu = ld<R>(U, V, mu, s);
  M3<double> v, gp;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const cx<R> e = mkc<R>(fmaR(coef, C.e[i].re, keep * Umu.e[i].re), fmaR(coef, C.e[i].im, keep * Umu.e[i].im));
    v.e[i] = mkc(to_f64(e.re), to_f64(e.im));
    gp.e[i] = mkc(to_f64(Gpm.e[i].re), to_f64(Gpm.e[i].im));
  }
  const M3<double> gv = project_su3_vjp_f64<sizeof(R) == 4 ? 1 : 2>(v, gp);
  const double kd = (double)keep, cd = (double)coef;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    gl.e[i] = mkc<R>(from_f64<R>(kd * gv.e[i].re), from_f64<R>(kd * gv.e[i].im));
    kk.e[i] = mkc<R>(from_f64<R>(cd * gv.e[i].re), from_f64<R>(cd * gv.e[i].im));
  }
}

// Gather stage for link (y, a), a in dirs: acc += sum_{mu in dirs, mu != a} [
//     K_mu(y) U_a(y+mu) U_mu(y+a)^dag + K_mu(y-mu)^dag U_a(y-mu) U_mu(y-mu+a)
//   + U_mu(y) U_a(y+mu) K_mu(y+a)^dag + U_mu(y-mu)^dag U_a(y-mu) K_mu(y-mu+a)
//   + U_mu(y-mu)^dag K_a(y-mu) U_mu(y-mu+a) + U_mu(y) K_a(y+mu) U_mu(y+a)^dag ]
// (10 products per mu: the common factors of the three terms through y+mu
// and of the three through y-mu are formed once).
template <typename R>
__device__ __forceinline__ void staple_gather(const V2<R>* __restrict__ U, const V2<R>* __restrict__ K,
                                              const GeomArgs& g, int s, const int c[4], int a, unsigned dirs,
                                              M3<R>& acc) {
  const long long V = g.V;
  const int s_pa = nb_fwd_rt(g, s, coord_of(c, a), a);
  // not unrolled: one copy of the ten products keeps the kernel's code small
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    if (mu == a || !((dirs >> mu) & 1u)) continue;
    const int cm = coord_of(c, mu);
    const int s_pmu = nb_fwd_rt(g, s, cm, mu);
    const int s_mmu = nb_bwd_rt(g, s, cm, mu);
    const int s_mmu_pa = nb_bwd_rt(g, s_pa, cm, mu);  // y - mu + a
    // the three terms through y+mu, with A = U_mu(y), B = U_a(y+mu):
    //   (K_mu(y) B + A K_a(y+mu)) U_mu(y+a)^dag + (A B) K_mu(y+a)^dag
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
}

// Where the gradient G' at U^(j+1) comes from, and what is done with it.
enum BwdSrc { kSrcLoad = 0, kSrcWilson = 1, kSrcGather = 2 };
enum BwdDst { kDstStout = 0, kDstApe = 1, kDstFinal = 2 };

template <typename R> struct BwdArgs {
  const V2<R>* Unext;  // U^(j+1): links of the Wilson seed or of the gather
  const V2<R>* Knext;  // K of step j+1 (gather)
  const V2<R>* Gin;    // the seed (load), or G_U(local) of step j+1 (gather)
  const V2<R>* Ucur;   // U^(j), input of step j (link stage); the thin links (final)
  V2<R>* Gout;         // G_U(local) of step j (link stage); G at the thin links (final, may be NULL)
  V2<R>* Kout;         // K of step j (link stage)
  V2<R>* Fout;         // force TA(G U^dag) at the thin links (final, may be NULL)
  GeomArgs g;
  int s_begin, s_end;  // the sites the kernel handles (the whole lattice: 0, V)
  R w0, w1;            // stout: rho; APE: 1 - alpha and the staple coefficient
  R mbeta3;            // Wilson seed: -beta / 3
  unsigned dirs;
};

// One thread per link; the four directions of a block of 128 sites run in
// consecutive CTAs, so the neighbour links and K that the gathers and staple
// sums of a site block share are read while still in L1/L2.
template <typename R, int SRC, int DST>
__global__ void __launch_bounds__(128) k_bwd_step(BwdArgs<R> p) {
  const GeomArgs& g = p.g;
  const long long V = g.V;
  const long long sl = p.s_begin + (long long)(blockIdx.x / 4) * blockDim.x + threadIdx.x;
  if (sl >= p.s_end) return;
  const int s = (int)sl;
  const int a = blockIdx.x % 4;
  const long long off = (long long)a * 9 * V + s;
  int c[4];
  site_coords(g, s, c);
  const bool smeared = (p.dirs >> a) & 1u;
  // G' = G at U^(j+1) for the link (s, a)
  M3<R> Gp;
  if (SRC == kSrcWilson) {
    Gp = m_rscale(staple_sum<R, true>(p.Unext, g, s, c, a, 15u), p.mbeta3);
  } else {
    Gp = ld_m3<R>(p.Gin + off, V);
    if (SRC == kSrcGather && smeared) staple_gather<R>(p.Unext, p.Knext, g, s, c, a, p.dirs, Gp);
  }
  if (DST == kDstFinal) {
    if (p.Gout) st_m3<R>(p.Gout + off, V, Gp);
    if (p.Fout) st_m3<R>(p.Fout + off, V, m_ta(mul_nd(Gp, ld_m3<R>(p.Ucur + off, V))));
    return;
  }
  if (!smeared) {  // not smeared: the gradient passes through
    st_m3<R>(p.Gout + off, V, Gp);
    return;
  }
  M3<R> gl, kk;
  if (DST == kDstStout) {
    StoutLinkPre<R> pre;
    stout_link_pre<R>(p.Ucur, g, s, c, a, p.dirs, p.w0, pre);
    stout_link_rest<R>(p.Ucur, g, s, a, p.w0, pre, Gp, gl, kk);
  } else {
    ape_link_grad<R>(p.Ucur, g, s, c, a, p.dirs, p.w0, p.w1, Gp, gl, kk);
  }
  st_m3<R>(p.Gout + off, V, gl);
  st_m3<R>(p.Kout + off, V, kk);
}

template <typename R, int SRC, int DST>
static lq_status launch_bwd_step(const BwdArgs<R>& p, cudaStream_t s) {
  const unsigned grid = (unsigned)((((long long)p.s_end - p.s_begin + 127) / 128) * 4);
  if (grid == 0) return LQ_OK;
  k_bwd_step<R, SRC, DST><<<grid, 128, 0, s>>>(p);
  return launch_check("k_bwd_step");
}

template <typename R, int DST>
static lq_status launch_bwd_src(int src, const BwdArgs<R>& p, cudaStream_t s) {
  if (src == kSrcLoad) return launch_bwd_step<R, kSrcLoad, DST>(p, s);
  if (src == kSrcWilson) return launch_bwd_step<R, kSrcWilson, DST>(p, s);
  return launch_bwd_step<R, kSrcGather, DST>(p, s);
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
  const size_t db = fb / 4;   // one direction's planes
  Bufs b;
  b.s = s;
  lq_status st;
  // a scratch link field whose unsmeared directions hold the thin links'
  // (step kernels never write those, so they stay valid in every buffer)
  auto alloc_links = [&](void** p) -> lq_status {
    lq_status st2 = scratch_alloc(p, fb, s, who);
    if (st2 != LQ_OK) return st2;
    b.own.push_back(*p);
    for (int mu = 0; mu < 4 && st2 == LQ_OK; ++mu)
      if (!((dirs >> mu) & 1u))
        st2 = cuda_check(cudaMemcpyAsync((char*)*p + mu * db, (const char*)thin->ptr + mu * db, db,
                                         cudaMemcpyDeviceToDevice, s),
                         who);
    return st2;
  };
  auto alloc = [&](void** p) -> lq_status {
    lq_status st2 = scratch_alloc(p, fb, s, who);
    if (st2 == LQ_OK) b.own.push_back(*p);
    return st2;
  };
  void* hyp_scratch = nullptr;   // decorated links and their gradients
  if (kind == Smearing::kHyp && n > 0) {
    if ((st = scratch_alloc(&hyp_scratch, kHypBwdPlanes * (fb / 4), s, who))) return st;
    b.own.push_back(hyp_scratch);
  }
  // recomputed fields follow the forward entry points' defaults (FP32 stout
  // links are re-projected)
  const TuneChoice tc = stout_default_choice(thin->prec);
  const int reproject = thin->prec == LQ_F32 ? 1 : 0;
  void* hyp_work = nullptr;
  // one step from `in` into `out` (distinct fields)
  auto step = [&](const void* in, void* out) -> lq_status {
    if (kind == Smearing::kStout)
      return stout_step_range(in, out, thin->geom, thin->prec, w, dirs, reproject, tc, 0, V, s);
    if (kind == Smearing::kApe) return ape_step(in, out, thin->geom, thin->prec, w, dirs, s);
    lq_status st2 = cuda_check(cudaMemcpyAsync(out, in, fb, cudaMemcpyDeviceToDevice, s), who);
    if (st2 != LQ_OK) return st2;
    return hyp_run_steps(out, hyp_work, hyp_scratch, thin->geom, thin->prec, fb, sa.a[0], sa.a[1], sa.a[2], 1, s);
  };
  if (kind == Smearing::kHyp && n > 0 && (st = alloc(&hyp_work))) return st;
  // checkpoints: ck[j] holds U^(j) for j % every == 0, j < n (ck[0] is the thin field itself)
  std::vector<const void*> ck(n + 1, nullptr);
  ck[0] = thin->ptr;
  for (int j = every; j < n; j += every) {
    void* p = nullptr;
    if ((st = alloc_links(&p))) return st;
    ck[j] = p;
  }
  // two fields for recomputed U^(j) (the one in use and the next), one for
  // the ping-pong of the recomputation
  void* rbuf[2] = {nullptr, nullptr};
  void* rtmp = nullptr;
  const bool need_u_n = !seed && n > 0;
  const bool recompute = every > 1 && n > 1;
  if ((need_u_n || recompute) && (st = alloc_links(&rbuf[0]))) return st;
  if (recompute && ((st = alloc_links(&rbuf[1])) || (st = alloc_links(&rtmp)))) return st;
  // U^(j0 + m) from src = U^(j0) into dst (m >= 1), through rtmp when m >= 2
  auto advance = [&](const void* src, void* dst, int m) -> lq_status {
    const void* in = src;
    for (int k = 0; k < m; ++k) {
      void* out = ((m - 1 - k) % 2 == 0) ? dst : rtmp;
      lq_status st2 = step(in, out);
      if (st2 != LQ_OK) return st2;
      in = out;
    }
    return LQ_OK;
  };
  for (int j = every; j < n; j += every)
    if ((st = advance(ck[j - every], (void*)ck[j], every))) return st;
  // U^(j) from the nearest checkpoint below it, into a buffer other than `keep`
  auto get_links = [&](int j, const void* keep) -> const void* {
    if (ck[j]) return ck[j];
    const int j0 = (j / every) * every;
    void* dst = rbuf[0] != keep ? rbuf[0] : rbuf[1];
    return advance(ck[j0], dst, j - j0) == LQ_OK ? dst : nullptr;
  };
  if (kind == Smearing::kHyp) {
    // the HYP force keeps its per-level kernels (hyp.cu): seed, steps, force
    void *Ga, *Gb;
    if ((st = alloc(&Ga)) || (st = alloc(&Gb))) return st;
    if (seed) {
      if ((st = cuda_check(cudaMemcpyAsync(Ga, seed->ptr, fb, cudaMemcpyDeviceToDevice, s), who))) return st;
    } else {
      const void* Un = thin->ptr;
      if (n > 0) {
        const int j0 = ((n - 1) / every) * every;
        if ((st = advance(ck[j0], rbuf[0], n - j0))) return st;
        Un = rbuf[0];
      }
      dim3 grid((unsigned)((V + 127) / 128), 4);
      k_wilson_grad<R><<<grid, 128, 0, s>>>((const V2<R>*)Un, (V2<R>*)Ga, g, (R)(-beta / 3.0));
      if ((st = launch_check("k_wilson_grad"))) return st;
    }
    for (int j = n - 1; j >= 0; --j) {
      const void* Uj = get_links(j, nullptr);
      if (!Uj) return LQ_ERR_CUDA;
      if ((st = hyp_backward_step(Uj, Ga, Gb, hyp_scratch, thin->geom, thin->prec, fb, sa.a[0], sa.a[1], sa.a[2], s)))
        return st;
      std::swap(Ga, Gb);
    }
    if (force) {
      dim3 grid((unsigned)((V + 255) / 256), 4);
      k_force<R><<<grid, 256, 0, s>>>((const V2<R>*)thin->ptr, (const V2<R>*)Ga, (V2<R>*)force->ptr, V);
      if ((st = launch_check("k_force"))) return st;
    }
    if (grad_out)
      if ((st = cuda_check(cudaMemcpyAsync(grad_out->ptr, Ga, fb, cudaMemcpyDeviceToDevice, s), who))) return st;
    return LQ_OK;
  }
  // stout and APE: one fused kernel per step (gather of step j + link stage of step j-1)
  int nd = 0;
  for (int mu = 0; mu < 4; ++mu) nd += (dirs >> mu) & 1u;
  BwdArgs<R> p{};
  p.g = g;
  p.s_begin = 0;
  p.s_end = (int)V;
  p.dirs = dirs;
  p.mbeta3 = (R)(-beta / 3.0);
  if (kind == Smearing::kStout) {
    p.w0 = (R)w;
  } else {
    p.w0 = (R)(1.0 - w);
    p.w1 = (R)(nd > 1 ? w / (2.0 * (nd - 1)) : 0.0);   // as in lq_ape_smear
  }
  const int dst_link = kind == Smearing::kStout ? kDstStout : kDstApe;
  int src = seed ? kSrcLoad : kSrcWilson;
  p.Gin = seed ? (const V2<R>*)seed->ptr : nullptr;
  if (need_u_n) {   // U^(n) for the Wilson seed
    const int j0 = ((n - 1) / every) * every;
    if ((st = advance(ck[j0], rbuf[0], n - j0))) return st;
    p.Unext = (const V2<R>*)rbuf[0];
  } else if (!seed) {
    p.Unext = (const V2<R>*)thin->ptr;   // n = 0: the seed at the thin links
  }
  void *Ga = nullptr, *Gb = nullptr, *Ka = nullptr, *Kb = nullptr;
  if (n > 0 && ((st = alloc(&Ga)) || (st = alloc(&Gb)) || (st = alloc(&Ka)) || (st = alloc(&Kb)))) return st;
  for (int j = n - 1; j >= 0; --j) {
    const void* Uj = get_links(j, p.Unext);
    if (!Uj) return LQ_ERR_CUDA;
    p.Ucur = (const V2<R>*)Uj;
    p.Gout = (V2<R>*)Ga;
    p.Kout = (V2<R>*)Ka;
    st = dst_link == kDstStout ? launch_bwd_src<R, kDstStout>(src, p, s) : launch_bwd_src<R, kDstApe>(src, p, s);
    if (st != LQ_OK) return st;
    // the next kernel gathers step j's K on U^(j)
    src = kSrcGather;
    p.Unext = (const V2<R>*)Uj;
    p.Knext = (const V2<R>*)Ka;
    p.Gin = (const V2<R>*)Ga;
    std::swap(Ga, Gb);
    std::swap(Ka, Kb);
  }
  p.Ucur = (const V2<R>*)thin->ptr;
  p.Gout = grad_out ? (V2<R>*)grad_out->ptr : nullptr;
  p.Kout = nullptr;
  p.Fout = force ? (V2<R>*)force->ptr : nullptr;
  return launch_bwd_src<R, kDstFinal>(src, p, s);
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

// One step of the stout force recursion on a site range (the building block
// of lq_stout_backward for callers that hold one part of a lattice).
template <typename R>
static lq_status backward_step_range(const lq_field* u_next, const lq_field* k_next, const lq_field* g_in,
                                     const lq_field* u_cur, lq_field* g_out, lq_field* k_out, lq_field* force_out,
                                     int source, double rho, double beta, unsigned dirs, long long s_begin,
                                     long long s_end, cudaStream_t s) {
  BwdArgs<R> p{};
  p.g = geom_args(u_cur->geom);
  p.s_begin = (int)s_begin;
  p.s_end = (int)s_end;
  p.dirs = dirs;
  p.w0 = (R)rho;
  p.mbeta3 = (R)(-beta / 3.0);
  p.Unext = u_next ? (const V2<R>*)u_next->ptr : nullptr;
  p.Knext = k_next ? (const V2<R>*)k_next->ptr : nullptr;
  p.Gin = g_in ? (const V2<R>*)g_in->ptr : nullptr;
  p.Ucur = (const V2<R>*)u_cur->ptr;
  p.Gout = g_out ? (V2<R>*)g_out->ptr : nullptr;
  p.Kout = k_out ? (V2<R>*)k_out->ptr : nullptr;
  p.Fout = force_out ? (V2<R>*)force_out->ptr : nullptr;
  const int src = source == LQ_BWD_SOURCE_WILSON ? kSrcWilson : (source == LQ_BWD_SOURCE_GIVEN ? kSrcLoad : kSrcGather);
  if (k_out) return launch_bwd_src<R, kDstStout>(src, p, s);
  return launch_bwd_src<R, kDstFinal>(src, p, s);
}

extern "C" lq_status lq_stout_backward_step(const lq_field* u_next, const lq_field* k_next, const lq_field* g_in,
                                            const lq_field* u_cur, lq_field* g_out, lq_field* k_out,
                                            lq_field* force_out, int source, double rho, double beta,
                                            unsigned dirs_mask, long long s_begin, long long s_end, void* stream) {
  clear_error();
  const char* who = "lq_stout_backward_step";
  lq_status st = check_links(u_cur, who);
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, who)) != LQ_OK) return st;
  if (source != LQ_BWD_SOURCE_WILSON && source != LQ_BWD_SOURCE_GIVEN && source != LQ_BWD_SOURCE_GATHER) {
    set_error("%s: source must be LQ_BWD_SOURCE_WILSON, _GIVEN or _GATHER", who);
    return LQ_ERR_ARG;
  }
  const bool need_u_next = source != LQ_BWD_SOURCE_GIVEN, need_k_next = source == LQ_BWD_SOURCE_GATHER,
             need_g_in = source != LQ_BWD_SOURCE_WILSON;
  if ((need_u_next && !u_next) || (need_k_next && !k_next) || (need_g_in && !g_in)) {
    set_error("%s: the source needs u_next (Wilson, gather), k_next (gather) and g_in (given, gather)", who);
    return LQ_ERR_ARG;
  }
  if (k_out ? (!g_out || force_out) : (!g_out && !force_out)) {
    set_error("%s: give g_out and k_out (a link stage), or g_out and/or force_out without k_out (the last step)",
              who);
    return LQ_ERR_ARG;
  }
  const lq_field* all[7] = {u_next, k_next, g_in, u_cur, g_out, k_out, force_out};
  for (const lq_field* f : all) {
    if (!f) continue;
    if (f->kind != LQ_LINKS || f->prec != u_cur->prec || !same_geom(f->geom, u_cur->geom)) {
      set_error("%s: every field must be LINKS of u_cur's geometry and precision", who);
      return LQ_ERR_GEOM;
    }
  }
  for (int i = 4; i < 7; ++i) {   // the outputs against every other argument
    if (!all[i]) continue;
    for (int k = 0; k < 7; ++k)
      if (k != i && all[k] && all[k]->ptr == all[i]->ptr) {
        set_error("%s: outputs must not alias each other or an input", who);
        return LQ_ERR_ARG;
      }
  }
  if (!(rho >= 0.0) || rho > 1e6 || !(beta == beta) || s_begin < 0 || s_end < s_begin ||
      s_end > u_cur->geom.volume) {
    set_error("%s: need finite rho >= 0, finite beta and 0 <= s_begin <= s_end <= volume", who);
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  if (u_cur->prec == LQ_F64)
    return backward_step_range<double>(u_next, k_next, g_in, u_cur, g_out, k_out, force_out, source, rho, beta,
                                       dirs_mask, s_begin, s_end, s);
  return backward_step_range<float>(u_next, k_next, g_in, u_cur, g_out, k_out, force_out, source, rho, beta,
                                    dirs_mask, s_begin, s_end, s);
}
