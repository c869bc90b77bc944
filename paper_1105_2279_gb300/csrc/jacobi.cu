// Jacobi smearing of a quark field (Winter, "Accelerating QDP++ using GPUs",
// Sec. 6, Listing 1): the paper's application.  Listing 1 evaluates five
// expressions per iteration (copy, the hopping term for the first and the
// other directions, the axpy, the final scaling), one kernel each; here one
// fused kernel per iteration forms
//   chi'(x) = scale * (s0(x) + kappa * sum_mu [U_mu(x) chi(x+mu) + U_mu(x-mu)^dag chi(x-mu)])
// with scale = 1/norm in the last iteration and 1 otherwise, for all spins of
// a site at once (the links are read once per site).
#include <cstddef>

#include "lq_internal.h"
#include "stout_core.cuh"

namespace lq {

// A link from the full [dir][9][V] layout, or (PACKED) from rows 0 and 1 in a
// [dir][6][V] copy with row 2 = conj(row 0 x row 1), exact for SU(3): 2/3 of
// the link bytes of this HBM-bound kernel for 18 complex multiply-adds.
template <typename R, bool PACKED>
__device__ __forceinline__ M3<R> jacobi_link(const typename vec2<R>::type* __restrict__ U, long long V, int mu,
                                             int s) {
  if (!PACKED) return ld_link<R>(U, V, mu, s);
  M3<R> m;
  const typename vec2<R>::type* p = U + (long long)mu * 6 * V + s;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const typename vec2<R>::type e = __ldg(p + (long long)c * V);
    m.e[c] = mkc<R>(e.x, e.y);
  }
  auto cross = [&](int a, int b, int c, int d) {
    const cx<R> t = cmul(m.e[c], m.e[d]);
    return cconj(cfma(m.e[a], m.e[b], mkc<R>(-t.re, -t.im)));
  };
  m.e[6] = cross(1, 5, 2, 4);
  m.e[7] = cross(2, 3, 0, 5);
  m.e[8] = cross(0, 4, 1, 3);
  return m;
}

template <typename R>
__global__ void k_pack12(const typename vec2<R>::type* __restrict__ U, typename vec2<R>::type* __restrict__ P,
                         long long V) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // over 4 dirs x 6 comps x V
  if (i >= 24 * V) return;
  const long long s = i % V, dc = i / V, mu = dc / 6, c = dc % 6;
  P[i] = U[(mu * 9 + c) * V + s];
}

// One site per (thread, k): a block of N_threads threads covers N_threads *
// N_site consecutive sites, site k * N_threads + tid of its range in round k
// (consecutive threads on consecutive sites in every round: coalesced).
template <typename R, int NSPIN, bool PACKED>
__device__ __forceinline__ void jacobi_site(const typename vec2<R>::type* __restrict__ U,
                                            const typename vec2<R>::type* __restrict__ chi,
                                            const typename vec2<R>::type* __restrict__ s0,
                                            typename vec2<R>::type* __restrict__ out, const GeomArgs& g, R kappa,
                                            R scale, unsigned dirs, int s) {
  typedef typename vec2<R>::type V2;
  const long long V = g.V;
  int c[4];
  site_coords(g, s, c);
  cx<R> h[NSPIN][3];
#pragma unroll
  for (int sp = 0; sp < NSPIN; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) h[sp][a] = mkc<R>(0, 0);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (!((dirs >> mu) & 1u)) continue;
    const int s_f = nb_fwd(g, s, c[mu], mu);
    const int s_b = nb_bwd(g, s, c[mu], mu);
    {
      // U_mu(x) chi(x+mu)
      const M3<R> u = jacobi_link<R, PACKED>(U, V, mu, s);
#pragma unroll
      for (int sp = 0; sp < NSPIN; ++sp) {
        cx<R> v[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const V2 e = __ldg(chi + (long long)(3 * sp + b) * V + s_f);
          v[b] = mkc<R>(e.x, e.y);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) h[sp][a] = cfma(u.e[3 * a + b], v[b], h[sp][a]);
      }
    }
    {
      // U_mu(x-mu)^dag chi(x-mu)
      const M3<R> u = jacobi_link<R, PACKED>(U, V, mu, s_b);
#pragma unroll
      for (int sp = 0; sp < NSPIN; ++sp) {
        cx<R> v[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const V2 e = __ldg(chi + (long long)(3 * sp + b) * V + s_b);
          v[b] = mkc<R>(e.x, e.y);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) h[sp][a] = cfma_cn(u.e[3 * b + a], v[b], h[sp][a]);
      }
    }
  }
#pragma unroll
  for (int sp = 0; sp < NSPIN; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long off = (long long)(3 * sp + a) * V + s;
      const V2 e = __ldg(s0 + off);
      V2 o;
      o.x = scale * fmaR(kappa, h[sp][a].re, (R)e.x);
      o.y = scale * fmaR(kappa, h[sp][a].im, (R)e.y);
      out[off] = o;
    }
}

template <typename R, int NSPIN, bool PACKED = false>
__global__ void __launch_bounds__(256) k_jacobi(const typename vec2<R>::type* __restrict__ U,
                                                const typename vec2<R>::type* __restrict__ chi,
                                                const typename vec2<R>::type* __restrict__ s0,
                                                typename vec2<R>::type* __restrict__ out, GeomArgs g, R kappa,
                                                R scale, unsigned dirs, int nsite) {
  const long long base = (long long)blockIdx.x * blockDim.x * nsite + threadIdx.x;
  for (int k = 0; k < nsite; ++k) {
    const long long sl = base + (long long)k * blockDim.x;
    if (sl >= g.V) return;
    jacobi_site<R, NSPIN, PACKED>(U, chi, s0, out, g, kappa, scale, dirs, (int)sl);
  }
}

template <typename R>
__global__ void k_scale(typename vec2<R>::type* __restrict__ f, long long n, R scale) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    typename vec2<R>::type e = f[i];
    e.x *= scale;
    e.y *= scale;
    f[i] = e;
  }
}

template <typename R>
static void launch_jacobi(int nspin, bool packed, const void* U, const void* in, const void* s0, void* out,
                          const GeomArgs& g, double kappa, double scale, unsigned dirs, const TuneChoice& tc,
                          cudaStream_t s) {
  typedef typename vec2<R>::type V2;
  const long long per_block = (long long)tc.block * tc.nsite;
  const unsigned grid = (unsigned)((g.V + per_block - 1) / per_block);
#define LQ_J(NS, PK)                                                                                          \
  k_jacobi<R, NS, PK><<<grid, tc.block, 0, s>>>((const V2*)U, (const V2*)in, (const V2*)s0, (V2*)out, g, \
                                                (R)kappa, (R)scale, dirs, tc.nsite)
  if (nspin == 4) {
    if (packed) LQ_J(4, true);
    else LQ_J(4, false);
  } else {
    if (packed) LQ_J(1, true);
    else LQ_J(1, false);
  }
#undef LQ_J
}

static lq_status launch_jacobi_prec(int prec, int nspin, bool packed, const void* U, const void* in, const void* s0,
                                    void* out, const GeomArgs& g, double kappa, double scale, unsigned dirs,
                                    const TuneChoice& tc, cudaStream_t s) {
  if (prec == LQ_F64) launch_jacobi<double>(nspin, packed, U, in, s0, out, g, kappa, scale, dirs, tc, s);
  else launch_jacobi<float>(nspin, packed, U, in, s0, out, g, kappa, scale, dirs, tc, s);
  return launch_check("lq_jacobi_smear kernel");
}

// Tuner key of the Jacobi kernel: one entry per field kind and link storage.
static const char* jacobi_kernel_key(int nspin, bool packed) {
  if (nspin == 4) return packed ? "jacobi_fermion_packed" : "jacobi_fermion";
  return packed ? "jacobi_vector_packed" : "jacobi_vector";
}

// The thread geometry of [W] Sec. 4.4 as the tuner's search space: every
// N_threads in {32, 64, 128, 256} x N_site in {1, 2, 4, 8}, each timed on two
// iterations into the work buffers (the caller's field is not touched).
static lq_status jacobi_autotune(int prec, int nspin, bool packed, const void* U, const void* chi, void* w0, void* w1,
                                 const GeomArgs& g, double kappa, unsigned dirs, cudaStream_t s, TuneChoice* best) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  lq_status st = LQ_OK;
  const int blocks[] = {32, 64, 128, 256};
  const int nsites[] = {1, 2, 4, 8};
  for (int b : blocks)
    for (int ns : nsites) {
      TuneChoice c;
      c.block = b;
      c.nsite = ns;
      c.variant = 1;
      if ((st = launch_jacobi_prec(prec, nspin, packed, U, chi, chi, w0, g, kappa, 1.0, dirs, c, s))) break;
      cudaEventRecord(e0, s);
      launch_jacobi_prec(prec, nspin, packed, U, w0, chi, w1, g, kappa, 1.0, dirs, c, s);
      launch_jacobi_prec(prec, nspin, packed, U, w1, chi, w0, g, kappa, 1.0, dirs, c, s);
      cudaEventRecord(e1, s);
      if ((st = cuda_check(cudaEventSynchronize(e1), "lq_jacobi_smear autotune timing"))) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        *best = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_jacobi_smear(const lq_field* links, lq_field* chi, double kappa, int n_iter, double norm,
                                     unsigned dirs_mask, void* stream) {
  return lq_jacobi_smear_ex(links, chi, kappa, n_iter, norm, dirs_mask, nullptr, stream);
}

extern "C" lq_status lq_jacobi_smear_ex(const lq_field* links, lq_field* chi, double kappa, int n_iter,
                                        double norm, unsigned dirs_mask, const lq_jacobi_opts* opts,
                                        void* stream) {
  clear_error();
  // fields past opts->struct_size read as 0 (callers built against the
  // smaller struct without the launch-shape fields keep working)
  const int osz = opts ? opts->struct_size : 0;
  const int min_sz = (int)(offsetof(lq_jacobi_opts, compress_links) + sizeof(int));
  if (opts && osz != 0 && osz < min_sz) {
    set_error("lq_jacobi_smear: opts->struct_size %d too small", osz);
    return LQ_ERR_ARG;
  }
  const bool packed = osz >= min_sz && opts->compress_links;
  const int want_block = osz >= (int)(offsetof(lq_jacobi_opts, block) + sizeof(int)) ? opts->block : 0;
  const int want_nsite =
      osz >= (int)(offsetof(lq_jacobi_opts, sites_per_thread) + sizeof(int)) ? opts->sites_per_thread : 0;
  if (want_block < 0 || want_block > 256 || (want_block % 32) != 0 || want_nsite < 0 || want_nsite > 64) {
    set_error("lq_jacobi_smear: block must be a multiple of 32 in [32, 256] (0: tuned/default) and "
              "sites_per_thread in [1, 64] (0: tuned/default)");
    return LQ_ERR_ARG;
  }
  lq_status st = check_links(links, "lq_jacobi_smear");
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_jacobi_smear")) != LQ_OK) return st;
  if (!chi || (chi->kind != LQ_COLOR_VECTOR && chi->kind != LQ_FERMION)) {
    set_error("lq_jacobi_smear: chi must be a COLOR_VECTOR or FERMION field");
    return chi ? LQ_ERR_GEOM : LQ_ERR_ARG;
  }
  if (!same_geom(chi->geom, links->geom) || chi->prec != links->prec) {
    set_error("lq_jacobi_smear: links and chi differ in geometry or precision");
    return LQ_ERR_GEOM;
  }
  if (n_iter < 0 || !(norm == norm) || norm == 0.0 || !(kappa == kappa)) {
    set_error("lq_jacobi_smear: n_iter >= 0, finite kappa and a finite non-zero norm are required");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  const GeomArgs g = geom_args(chi->geom);
  const int nspin = chi->kind == LQ_FERMION ? 4 : 1;
  if (n_iter == 0) {
    const long long n = g.V * 3 * nspin;
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 8);
    if (chi->prec == LQ_F64)
      k_scale<double><<<grid, 256, 0, s>>>((double2*)chi->ptr, n, 1.0 / norm);
    else
      k_scale<float><<<grid, 256, 0, s>>>((float2*)chi->ptr, n, (float)(1.0 / norm));
    return launch_check("lq_jacobi_smear scale");
  }
  // chi stays s0 until the end; iterations ping-pong between two work buffers
  void* w[2] = {nullptr, nullptr};
  void* pk = nullptr;
  if ((st = scratch_alloc(&w[0], chi->bytes, s, "lq_jacobi_smear"))) return st;
  if ((st = scratch_alloc(&w[1], chi->bytes, s, "lq_jacobi_smear"))) {
    scratch_free(w[0], s);
    return st;
  }
  const void* U = links->ptr;
  if (packed) {   // rows 0 and 1 of every link, once for all iterations
    st = scratch_alloc(&pk, links->bytes / 9 * 6, s, "lq_jacobi_smear packed links");
    if (st == LQ_OK) {
      const long long n = 24 * g.V;
      const unsigned grid = (unsigned)((n + 255) / 256);
      if (chi->prec == LQ_F64)
        k_pack12<double><<<grid, 256, 0, s>>>((const double2*)links->ptr, (double2*)pk, g.V);
      else
        k_pack12<float><<<grid, 256, 0, s>>>((const float2*)links->ptr, (float2*)pk, g.V);
      st = launch_check("lq_jacobi_smear pack");
      U = pk;
    }
  }
  // thread geometry: explicit, else tuned (when the tuner is on), else 128 x 1
  TuneChoice tc;
  tc.block = 128;
  tc.nsite = 1;
  tc.variant = 1;
  if (want_block > 0 || want_nsite > 0) {
    if (want_block > 0) tc.block = want_block;
    if (want_nsite > 0) tc.nsite = want_nsite;
  } else if (st == LQ_OK && tune_enabled()) {
    const char* key = jacobi_kernel_key(nspin, packed);
    if (!tune_get(key, chi->prec, chi->geom.dims, dirs_mask, &tc)) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(s, &cs);
      if (cs == cudaStreamCaptureStatusNone) {   // never tune inside a capture
        st = jacobi_autotune(chi->prec, nspin, packed, U, chi->ptr, w[0], w[1], g, kappa, dirs_mask, s, &tc);
        if (st == LQ_OK) tune_put(key, chi->prec, chi->geom.dims, dirs_mask, tc);
      }
    }
  }
  const void* cur = chi->ptr;
  for (int it = 0; it < n_iter && st == LQ_OK; ++it) {
    void* out = w[it & 1];
    const double scale = (it == n_iter - 1) ? 1.0 / norm : 1.0;
    st = launch_jacobi_prec(chi->prec, nspin, packed, U, cur, chi->ptr, out, g, kappa, scale, dirs_mask, tc, s);
    cur = out;
  }
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpyAsync(chi->ptr, cur, chi->bytes, cudaMemcpyDeviceToDevice, s), "lq_jacobi_smear copy");
  scratch_free(w[0], s);
  scratch_free(w[1], s);
  if (pk) scratch_free(pk, s);
  return st;
}
