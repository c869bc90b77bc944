// Stout link smearing: one fused kernel per step (staples -> Omega -> Q ->
// FP64 Cayley-Hamilton coefficients -> exp(iQ) U -> optional FP64
// re-projection), double-buffered over n steps, optionally replayed as a
// CUDA graph (Morningstar & Peardon 2004, Secs. II-III; thread geometry
// N_threads / N_site of Winter, "Accelerating QDP++ using GPUs", Sec. 4.4).
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "lq_internal.h"
#include "stout_core.cuh"

namespace lq {

struct MuList {
  int mu[4];
};

// Variant 1: one thread per (site, mu) for N_site sites; neighbour links are
// read through the read-only data path (L1 / L2 serve the ~19x reuse of each
// link by neighbouring staples).  Consecutive blocks take the smeared
// directions of one site block, so the four sweeps share cached lines and
// the field streams from DRAM about once per step.
// With COUNT, every warp adds to stats[0..2] its link updates, those whose
// coefficients took the series, and the sum of their series orders K.
__device__ __forceinline__ void count_series(unsigned long long* stats, int k) {
  const unsigned m = __activemask();
  const unsigned n_series = __reduce_add_sync(m, k > 0 ? 1u : 0u);
  const unsigned sum_k = __reduce_add_sync(m, (unsigned)k);
  if ((int)(threadIdx.x & 31) == __ffs(m) - 1) {
    atomicAdd(&stats[0], (unsigned long long)__popc(m));
    atomicAdd(&stats[1], (unsigned long long)n_series);
    atomicAdd(&stats[2], (unsigned long long)sum_k);
  }
}

// Sites [s_begin, s_end) of the lattice (the whole lattice, or one slab of
// t-slices when the host-streamed path smears slab by slab).
template <typename R, bool REPRO, bool COUNT>
__device__ __forceinline__ void stout_global_body(const typename vec2<R>::type* __restrict__ Uin,
                                                  typename vec2<R>::type* __restrict__ Uout, const GeomArgs& g,
                                                  R rho, unsigned dirs, int nsite, int nd, const MuList& ml,
                                                  unsigned long long* stats, int s_begin, int s_end,
                                                  int blk) {
  const int mi = blk % nd;
  const long long sb = blk / nd;
  const int mu = mi == 0 ? ml.mu[0] : (mi == 1 ? ml.mu[1] : (mi == 2 ? ml.mu[2] : ml.mu[3]));
  const long long V = g.V;
  for (int k = 0; k < nsite; ++k) {
    const long long sl = s_begin + (sb * nsite + k) * blockDim.x + threadIdx.x;
    if (sl >= s_end) return;
    const int s = (int)sl;
    int c[4];
    site_coords(g, s, c);
    int korder = 0;
    const M3<R> Up = stout_link<R>(Uin, g, s, c, mu, dirs, rho, REPRO, COUNT ? &korder : nullptr);
    st_m3<R>(Uout + (long long)mu * 9 * V + s, V, Up);
    if (COUNT) count_series(stats, korder);
  }
}

// FP32 links: capped at 80 registers (16 bytes of spill), 24 resident warps
// per SM for blocks of 128 or 256 threads: measured against 72 (28 warps,
// 168 bytes of spill) and 96 (20 warps, none) at 48^3x96, 8.08 ms per step
// against 8.14 and 8.33.
template <bool REPRO, bool COUNT = false>
__global__ void __maxnreg__(80) k_stout_global_f32(const float2* __restrict__ Uin, float2* __restrict__ Uout,
                                                   GeomArgs g, float rho, unsigned dirs, int nsite, int nd,
                                                   MuList ml, unsigned long long* stats, int s_begin, int s_end) {
  stout_global_body<float, REPRO, COUNT>(Uin, Uout, g, rho, dirs, nsite, nd, ml, stats, s_begin, s_end, blockIdx.x);
}

template <bool REPRO, bool COUNT = false>
__global__ void __launch_bounds__(256) k_stout_global_f64(const double2* __restrict__ Uin,
                                                          double2* __restrict__ Uout, GeomArgs g, double rho,
                                                          unsigned dirs, int nsite, int nd, MuList ml,
                                                          unsigned long long* stats, int s_begin, int s_end) {
  stout_global_body<double, REPRO, COUNT>(Uin, Uout, g, rho, dirs, nsite, nd, ml, stats, s_begin, s_end,
                                          blockIdx.x);
}

// Several independent site ranges, each with its own input and output field,
// in one launch (the host-streamed path runs the (step, slab) items of one
// wavefront key together: one grid tail instead of one per slab).
struct SegList {
  const void* in[kMaxSegs];
  void* out[kMaxSegs];
  int s0[kMaxSegs], s1[kMaxSegs];
  int bstart[kMaxSegs + 1];   // first block of each segment; bstart[n] = grid size
  int n;
};

template <typename R, bool REPRO>
__device__ __forceinline__ void stout_seg_body(const SegList& sg, GeomArgs g, R rho, unsigned dirs, int nsite,
                                               int nd, MuList ml) {
  int j = 0;
#pragma unroll 1
  while (j + 1 < sg.n && (int)blockIdx.x >= sg.bstart[j + 1]) ++j;
  typedef typename vec2<R>::type V2;
  stout_global_body<R, REPRO, false>((const V2*)sg.in[j], (V2*)sg.out[j], g, rho, dirs, nsite, nd, ml, nullptr,
                                     sg.s0[j], sg.s1[j], (int)blockIdx.x - sg.bstart[j]);
}

template <bool REPRO>
__global__ void __maxnreg__(80) k_stout_seg_f32(SegList sg, GeomArgs g, float rho, unsigned dirs, int nsite, int nd,
                                                MuList ml) {
  stout_seg_body<float, REPRO>(sg, g, rho, dirs, nsite, nd, ml);
}

template <bool REPRO>
__global__ void __launch_bounds__(256) k_stout_seg_f64(SegList sg, GeomArgs g, double rho, unsigned dirs, int nsite,
                                                       int nd, MuList ml) {
  stout_seg_body<double, REPRO>(sg, g, rho, dirs, nsite, nd, ml);
}

// Variant 2 (FP32): shared-memory staging.  A CTA owns a BX x BY x BZ block of
// (x, y, z) and marches along t over `tchunk` slices, keeping a ring of three
// t-slices (t-1, t, t+1) of all four link directions on the block plus a
// one-site halo in shared memory; every staple link then comes from shared
// memory.  The arithmetic and its order equal variant 1, so results are
// bit-identical.
constexpr int kSmemBX = 4, kSmemBY = 4, kSmemBZ = 4;
constexpr int kSmemThreads = kSmemBX * kSmemBY * kSmemBZ * 4;
constexpr int kSmemHS = (kSmemBX + 2) * (kSmemBY + 2) * (kSmemBZ + 2);

template <typename R>
__device__ __forceinline__ M3<R> sm_link(const typename vec2<R>::type* __restrict__ slot_base, int dir, int h) {
  M3<R> m;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const typename vec2<R>::type v = slot_base[(dir * 9 + c) * kSmemHS + h];
    m.e[c].re = v.x;
    m.e[c].im = v.y;
  }
  return m;
}

template <typename R, bool REPRO>
__global__ void __launch_bounds__(kSmemThreads, 1) k_stout_smem(const typename vec2<R>::type* __restrict__ Uin,
                                                                 typename vec2<R>::type* __restrict__ Uout,
                                                                 GeomArgs g, R rho, unsigned dirs, int nd,
                                                                 MuList ml, int tchunk) {
  typedef typename vec2<R>::type V2;
  constexpr int BX = kSmemBX, BY = kSmemBY, BZ = kSmemBZ, HX = BX + 2, HY = BY + 2, HS = kSmemHS;
  constexpr int NB = BX * BY * BZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2* sm = reinterpret_cast<V2*>(smem_raw);  // [3 slots][36 planes][HS]
  const int ntx = (g.L[0] + BX - 1) / BX, nty = (g.L[1] + BY - 1) / BY, ntz = (g.L[2] + BZ - 1) / BZ;
  int b = blockIdx.x;
  const int x0 = (b % ntx) * BX;
  b /= ntx;
  const int y0 = (b % nty) * BY;
  b /= nty;
  const int z0 = (b % ntz) * BZ;
  b /= ntz;
  const int t0 = b * tchunk;
  const int t1 = min(t0 + tchunk, g.L[3]);
  const int tid = threadIdx.x;
  const int mi = tid / NB, ls = tid % NB;
  const int lx = ls % BX, ly = (ls / BX) % BY, lz = ls / (BX * BY);
  const long long V = g.V;
  const int mu = mi == 0 ? ml.mu[0] : (mi == 1 ? ml.mu[1] : (mi == 2 ? ml.mu[2] : ml.mu[3]));
  const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
  const bool active = mi < nd && x < g.L[0] && y < g.L[1] && z < g.L[2];
  // halo index of this thread's site and the unit steps along x, y, z
  const int hc = (lx + 1) + HX * ((ly + 1) + HY * (lz + 1));

  auto load_slice = [&](int t) {  // t in [-1, Lt]; periodic
    const int tw = (t + g.L[3]) % g.L[3];
    V2* dst = sm + (size_t)((t + 3) % 3) * 36 * HS;
    for (int i = tid; i < 36 * HS; i += kSmemThreads) {
      const int p = i / HS, h = i - p * HS;
      const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
      const int gx = (x0 - 1 + hx + g.L[0]) % g.L[0];
      const int gy = (y0 - 1 + hy + g.L[1]) % g.L[1];
      const int gz = (z0 - 1 + hz + g.L[2]) % g.L[2];
      dst[i] = __ldg(Uin + (long long)p * V + (gx + g.L[0] * (gy + g.L[1] * (gz + g.L[2] * tw))));
    }
  };
  // link `dir` at the site displaced by (+-1 along a, +-1 along b) from this thread's site
  auto link = [&](int t, int dir, int a, int da, int bdir, int db) -> M3<R> {
    int h = hc, dt = 0;
    if (a == 3) dt += da; else h += da * (a == 0 ? 1 : (a == 1 ? HX : HX * HY));
    if (bdir == 3) dt += db; else h += db * (bdir == 0 ? 1 : (bdir == 1 ? HX : HX * HY));
    return sm_link<R>(sm + (size_t)((t + dt + 3) % 3) * 36 * HS, dir, h);
  };

  for (int t = t0; t < t1; ++t) {
    if (t == t0) {
      load_slice(t - 1);
      load_slice(t);
    }
    load_slice(t + 1);
    __syncthreads();
    if (active) {
      M3<R> S;
      m_zero(S);
#pragma unroll
      for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu || !((dirs >> nu) & 1u)) continue;
        {
          // U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
          M3<R> tmp = mul_nd(link(t, mu, nu, 1, nu, 0), link(t, nu, mu, 1, mu, 0));
          mac_nn(S, link(t, nu, nu, 0, nu, 0), tmp);
        }
        {
          // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
          M3<R> tmp = mul_nn(link(t, mu, nu, -1, nu, 0), link(t, nu, nu, -1, mu, 1));
          mac_dn(S, link(t, nu, nu, -1, nu, 0), tmp);
        }
      }
      const M3<R> Up = stout_update<R>(S, link(t, mu, mu, 0, mu, 0), rho, REPRO);
      const int s = x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
      st_m3<R>(Uout + (long long)mu * 9 * V + s, V, Up);
    }
    __syncthreads();
  }
}

static size_t smem_bytes_f32() { return (size_t)3 * 36 * kSmemHS * sizeof(float2); }

// Variant 3: two kernels per step.  The two-link products
//   W_{mu nu}(y) = U_mu(y) U_nu(y + mu)
// of every ordered pair of smeared directions are formed once per step (one
// product each), and each serves two staples:
//   upper staple of (x, mu) in plane nu = W_{nu mu}(x) U_nu(x + mu)^dag
//   lower staple of (x, mu) in plane nu = U_nu(x - nu)^dag W_{mu nu}(x - nu)
// so a link's six staples cost 6 + 3 products (3 W per link on average)
// instead of 12, for W read and written through HBM.  For FP64 links,
// whose step is bound by the FP64 pipe.
struct PairMap {
  int idx[16];   // idx[4 mu + nu]: W plane of the ordered pair (mu, nu), -1 if unused
  int mu[12], nu[12];
  int n;
};

static PairMap pair_map(unsigned dirs) {
  PairMap pm;
  pm.n = 0;
  for (int i = 0; i < 16; ++i) pm.idx[i] = -1;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      if (a != b && ((dirs >> a) & 1u) && ((dirs >> b) & 1u)) {
        pm.idx[4 * a + b] = pm.n;
        pm.mu[pm.n] = a;
        pm.nu[pm.n] = b;
        ++pm.n;
      }
  return pm;
}

static size_t wfield_bytes(const lq_geom& g, int prec, unsigned dirs) {
  return (size_t)pair_map(dirs).n * 9 * (size_t)g.volume * elem_bytes(LQ_LINKS, prec);
}

template <typename R>
__global__ void __launch_bounds__(128) k_wfield(const typename vec2<R>::type* __restrict__ U,
                                                typename vec2<R>::type* __restrict__ W, GeomArgs g, PairMap pm) {
  // the pairs of one site block run in consecutive CTAs, so their reads of
  // the same links hit in L2 (a pair-major grid re-read the lattice per pair)
  const long long V = g.V;
  const int p = blockIdx.x % pm.n;
  const long long sl = (long long)(blockIdx.x / pm.n) * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const int s = (int)sl;
  const int mu = pm.mu[p], nu = pm.nu[p];
  int c[4];
  site_coords(g, s, c);
  const int s_pmu = nb_fwd(g, s, coord_of(c, mu), mu);
  st_m3<R>(W + (long long)p * 9 * V + s, V, mul_nn(ld_link<R>(U, V, mu, s), ld_link<R>(U, V, nu, s_pmu)));
}

template <typename R, bool REPRO>
__global__ void __launch_bounds__(256) k_stout_wf(const typename vec2<R>::type* __restrict__ Uin,
                                                  const typename vec2<R>::type* __restrict__ W,
                                                  typename vec2<R>::type* __restrict__ Uout, GeomArgs g, R rho,
                                                  unsigned dirs, int nd, MuList ml, PairMap pm) {
  const int mi = blockIdx.x % nd;
  const long long sl = (long long)(blockIdx.x / nd) * blockDim.x + threadIdx.x;
  const long long V = g.V;
  if (sl >= V) return;
  const int mu = mi == 0 ? ml.mu[0] : (mi == 1 ? ml.mu[1] : (mi == 2 ? ml.mu[2] : ml.mu[3]));
  const int s = (int)sl;
  int c[4];
  site_coords(g, s, c);
  const int s_pmu = nb_fwd(g, s, coord_of(c, mu), mu);
  M3<R> S;
  m_zero(S);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu || !((dirs >> nu) & 1u)) continue;
    const int cn = coord_of(c, nu);
    const int Ln = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
    const int sn = nu == 0 ? g.stride[0] : (nu == 1 ? g.stride[1] : (nu == 2 ? g.stride[2] : g.stride[3]));
    const int s_mnu = (cn > 0) ? s - sn : s + (Ln - 1) * sn;
    const int p_up = pm.idx[4 * nu + mu], p_lo = pm.idx[4 * mu + nu];
    mac_nd(S, ld_m3<R>(W + (long long)p_up * 9 * V + s, V), ld_link<R>(Uin, V, nu, s_pmu));
    mac_dn(S, ld_link<R>(Uin, V, nu, s_mnu), ld_m3<R>(W + (long long)p_lo * 9 * V + s_mnu, V));
  }
  const M3<R> Up = stout_update<R>(S, ld_link<R>(Uin, V, mu, s), rho, REPRO);
  st_m3<R>(Uout + (long long)mu * 9 * V + s, V, Up);
}

static MuList mu_list(unsigned dirs, int* n) {
  MuList m;
  int k = 0;
  for (int mu = 0; mu < 4; ++mu)
    if ((dirs >> mu) & 1u) m.mu[k++] = mu;
  for (int j = k; j < 4; ++j) m.mu[j] = 0;
  *n = k;
  return m;
}

// One step on the global-load kernel over sites [s_begin, s_end).
static lq_status launch_global(const void* in, void* out, const GeomArgs& g, int prec, double rho, unsigned dirs,
                               int reproject, const TuneChoice& tc, long long s_begin, long long s_end,
                               cudaStream_t s) {
  int nd = 0;
  const MuList ml = mu_list(dirs, &nd);
  const int block = tc.block > 0 ? tc.block : 128;
  const int nsite = tc.nsite > 0 ? tc.nsite : 1;
  const long long per_block = (long long)block * nsite;
  const int sb = (int)s_begin, se = (int)s_end;
  dim3 grid((unsigned)(((s_end - s_begin + per_block - 1) / per_block) * nd));
  if (grid.x == 0) return LQ_OK;
  if (prec == LQ_F64) {
    if (reproject)
      k_stout_global_f64<true><<<grid, block, 0, s>>>((const double2*)in, (double2*)out, g, rho, dirs, nsite, nd, ml,
                                                      nullptr, sb, se);
    else
      k_stout_global_f64<false><<<grid, block, 0, s>>>((const double2*)in, (double2*)out, g, rho, dirs, nsite, nd,
                                                       ml, nullptr, sb, se);
  } else {
    if (reproject)
      k_stout_global_f32<true><<<grid, block, 0, s>>>((const float2*)in, (float2*)out, g, (float)rho, dirs, nsite, nd,
                                                      ml, nullptr, sb, se);
    else
      k_stout_global_f32<false><<<grid, block, 0, s>>>((const float2*)in, (float2*)out, g, (float)rho, dirs, nsite,
                                                       nd, ml, nullptr, sb, se);
  }
  return launch_check("stout step kernel");
}

lq_status stout_step_range(const void* in, void* out, const lq_geom& geom, int prec, double rho, unsigned dirs,
                           int reproject, const TuneChoice& tc, long long s_begin, long long s_end, cudaStream_t s) {
  TuneChoice t = tc;
  if (t.variant != 1) t = stout_default_choice(prec);   // variants 2 and 3 work on whole lattices
  return launch_global(in, out, geom_args(geom), prec, rho, dirs, reproject, t, s_begin, s_end, s);
}

lq_status stout_step_segments(const StepSegment* seg, int nseg, const lq_geom& geom, int prec, double rho,
                              unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s) {
  TuneChoice t = tc;
  if (t.variant != 1) t = stout_default_choice(prec);
  const GeomArgs g = geom_args(geom);
  int nd = 0;
  const MuList ml = mu_list(dirs, &nd);
  const int block = t.block > 0 ? t.block : 128;
  const int nsite = t.nsite > 0 ? t.nsite : 1;
  const long long per_block = (long long)block * nsite;
  for (int first = 0; first < nseg; first += kMaxSegs) {
    SegList sl;
    sl.n = nseg - first < kMaxSegs ? nseg - first : kMaxSegs;
    long long b = 0;
    for (int j = 0; j < sl.n; ++j) {
      const StepSegment& e = seg[first + j];
      sl.in[j] = e.in;
      sl.out[j] = e.out;
      sl.s0[j] = (int)e.s_begin;
      sl.s1[j] = (int)e.s_end;
      sl.bstart[j] = (int)b;
      b += ((e.s_end - e.s_begin + per_block - 1) / per_block) * nd;
    }
    sl.bstart[sl.n] = (int)b;
    for (int j = sl.n + 1; j <= kMaxSegs; ++j) sl.bstart[j] = (int)b;
    if (b == 0) continue;
    if (prec == LQ_F64) {
      if (reproject) k_stout_seg_f64<true><<<(unsigned)b, block, 0, s>>>(sl, g, rho, dirs, nsite, nd, ml);
      else k_stout_seg_f64<false><<<(unsigned)b, block, 0, s>>>(sl, g, rho, dirs, nsite, nd, ml);
    } else {
      if (reproject) k_stout_seg_f32<true><<<(unsigned)b, block, 0, s>>>(sl, g, (float)rho, dirs, nsite, nd, ml);
      else k_stout_seg_f32<false><<<(unsigned)b, block, 0, s>>>(sl, g, (float)rho, dirs, nsite, nd, ml);
    }
    lq_status st = launch_check("stout step kernel (segments)");
    if (st != LQ_OK) return st;
  }
  return LQ_OK;
}

static lq_status launch_step(const void* in, void* out, const lq_geom& geom, int prec, double rho,
                             unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s,
                             void* wbuf = nullptr) {
  const GeomArgs g = geom_args(geom);
  int nd = 0;
  const MuList ml = mu_list(dirs, &nd);
  if (tc.variant == 3 && wbuf) {
    const PairMap pm = pair_map(dirs);
    const unsigned gs = (unsigned)((g.V + 127) / 128 * pm.n);
    const int block = tc.block > 0 ? tc.block : 128;
    const dim3 grid((unsigned)(((g.V + block - 1) / block) * nd));
    if (prec == LQ_F64) {
      k_wfield<double><<<gs, 128, 0, s>>>((const double2*)in, (double2*)wbuf, g, pm);
      if (reproject)
        k_stout_wf<double, true><<<grid, block, 0, s>>>((const double2*)in, (const double2*)wbuf, (double2*)out, g,
                                                        rho, dirs, nd, ml, pm);
      else
        k_stout_wf<double, false><<<grid, block, 0, s>>>((const double2*)in, (const double2*)wbuf, (double2*)out, g,
                                                         rho, dirs, nd, ml, pm);
    } else {
      k_wfield<float><<<gs, 128, 0, s>>>((const float2*)in, (float2*)wbuf, g, pm);
      if (reproject)
        k_stout_wf<float, true><<<grid, block, 0, s>>>((const float2*)in, (const float2*)wbuf, (float2*)out, g,
                                                       (float)rho, dirs, nd, ml, pm);
      else
        k_stout_wf<float, false><<<grid, block, 0, s>>>((const float2*)in, (const float2*)wbuf, (float2*)out, g,
                                                        (float)rho, dirs, nd, ml, pm);
    }
    return launch_check("stout step kernels (two-link product variant)");
  }
  if (tc.variant == 2 && prec == LQ_F32) {
    static bool attr_set[64] = {false};
    const int dev = current_device();
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
      lq_status st = cuda_check(cudaFuncSetAttribute(k_stout_smem<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem_bytes_f32()), "stout smem attribute");
      if (st == LQ_OK)
        st = cuda_check(cudaFuncSetAttribute(k_stout_smem<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes_f32()), "stout smem attribute");
      if (st != LQ_OK) return st;
      attr_set[dev] = true;
    }
    const int tchunk = tc.nsite > 0 ? tc.nsite : 8;
    const long long ntiles = (long long)((g.L[0] + kSmemBX - 1) / kSmemBX) * ((g.L[1] + kSmemBY - 1) / kSmemBY) *
                             ((g.L[2] + kSmemBZ - 1) / kSmemBZ) * ((g.L[3] + tchunk - 1) / tchunk);
    if (reproject)
      k_stout_smem<float, true><<<(unsigned)ntiles, kSmemThreads, smem_bytes_f32(), s>>>(
          (const float2*)in, (float2*)out, g, (float)rho, dirs, nd, ml, tchunk);
    else
      k_stout_smem<float, false><<<(unsigned)ntiles, kSmemThreads, smem_bytes_f32(), s>>>(
          (const float2*)in, (float2*)out, g, (float)rho, dirs, nd, ml, tchunk);
    return launch_check("stout step kernel (shared-memory variant)");
  }
  return launch_global(in, out, g, prec, rho, dirs, reproject, tc, 0, g.V, s);
}

static size_t dir_block_bytes(const lq_geom& g, int prec) {
  return (size_t)g.volume * 9 * elem_bytes(LQ_LINKS, prec);
}

static lq_status stout_run_steps_impl(void* links, void* work, const lq_geom& g, int prec, double rho, int n_steps,
                                      unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s, void* wbuf);

lq_status stout_run_steps(void* links, void* work, const lq_geom& g, int prec, double rho, int n_steps,
                          unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s, void* wbuf) {
  if (n_steps <= 0) return LQ_OK;
  void* own_w = nullptr;
  if (tc.variant == 3 && !wbuf) {
    lq_status st = scratch_alloc(&own_w, wfield_bytes(g, prec, dirs), s, "stout two-link products");
    if (st != LQ_OK) return st;
    wbuf = own_w;
  }
  lq_status st = stout_run_steps_impl(links, work, g, prec, rho, n_steps, dirs, reproject, tc, s, wbuf);
  if (own_w) scratch_free(own_w, s);
  return st;
}

static lq_status stout_run_steps_impl(void* links, void* work, const lq_geom& g, int prec, double rho, int n_steps,
                                      unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s, void* wbuf) {
  const size_t db = dir_block_bytes(g, prec);
  // links outside `dirs` are never written: give the work buffer a copy once
  for (int mu = 0; mu < 4; ++mu)
    if (!((dirs >> mu) & 1u)) {
      lq_status st = cuda_check(cudaMemcpyAsync((char*)work + mu * db, (const char*)links + mu * db, db,
                                                cudaMemcpyDeviceToDevice, s),
                                "stout pass-through copy");
      if (st != LQ_OK) return st;
    }
  for (int k = 0; k < n_steps; ++k) {
    const void* in = (k % 2 == 0) ? links : work;
    void* out = (k % 2 == 0) ? work : links;
    lq_status st = launch_step(in, out, g, prec, rho, dirs, reproject, tc, s, wbuf);
    if (st != LQ_OK) return st;
  }
  if (n_steps % 2 == 1) {
    for (int mu = 0; mu < 4; ++mu)
      if ((dirs >> mu) & 1u) {
        lq_status st = cuda_check(cudaMemcpyAsync((char*)links + mu * db, (const char*)work + mu * db, db,
                                                  cudaMemcpyDeviceToDevice, s),
                                  "stout result copy");
        if (st != LQ_OK) return st;
      }
  }
  return LQ_OK;
}

TuneChoice stout_default_choice(int prec) {
  TuneChoice c;
  c.block = 128;
  c.nsite = 1;
  c.variant = 1;
  (void)prec;
  return c;
}

// Times one step of every candidate on a scratch output (links untouched).
static lq_status stout_autotune(const lq_field* f, double rho, unsigned dirs, int reproject, cudaStream_t s,
                                TuneChoice* best) {
  void* tmp = nullptr;
  lq_status st = scratch_alloc(&tmp, f->bytes, s, "stout autotune");
  if (st != LQ_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  *best = stout_default_choice(f->prec);
  const int blocks[] = {64, 128, 256};
  const int nsites[] = {1, 2, 4};
  for (int b : blocks)
    for (int ns : nsites) {
      TuneChoice c;
      c.block = b;
      c.nsite = ns;
      c.variant = 1;
      st = launch_step(f->ptr, tmp, f->geom, f->prec, rho, dirs, reproject, c, s);  // warm-up
      if (st != LQ_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 2; ++r) launch_step(f->ptr, tmp, f->geom, f->prec, rho, dirs, reproject, c, s);
      cudaEventRecord(e1, s);
      st = cuda_check(cudaEventSynchronize(e1), "stout autotune timing");
      if (st != LQ_OK) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        *best = c;
      }
    }
  if (st == LQ_OK && f->prec == LQ_F32) {
    const int tchunks[] = {4, 8, 16};
    for (int tcn : tchunks) {
      TuneChoice c;
      c.block = kSmemThreads;
      c.nsite = tcn;
      c.variant = 2;
      st = launch_step(f->ptr, tmp, f->geom, f->prec, rho, dirs, reproject, c, s);
      if (st != LQ_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 2; ++r) launch_step(f->ptr, tmp, f->geom, f->prec, rho, dirs, reproject, c, s);
      cudaEventRecord(e1, s);
      st = cuda_check(cudaEventSynchronize(e1), "stout autotune timing");
      if (st != LQ_OK) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        *best = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch_free(tmp, s);
  return st;
}

lq_status stout_choose(const lq_field* f, double rho, unsigned dirs, int reproject, const lq_stout_opts* o,
                       cudaStream_t s, TuneChoice* out) {
  if (o && (o->block > 0 || o->variant > 0)) {  // explicit launch shape
    out->variant = o->variant > 0 ? o->variant : 1;
    if (out->variant == 2) {
      out->block = kSmemThreads;
      out->nsite = o->sites_per_thread > 0 ? o->sites_per_thread : 8;  // t-slices per CTA
    } else if (out->variant == 3) {
      out->block = o->block > 0 ? o->block : 128;
      out->nsite = 1;
    } else {
      out->block = o->block > 0 ? o->block : 128;
      out->nsite = o->sites_per_thread > 0 ? o->sites_per_thread : 1;
    }
    return LQ_OK;
  }
  *out = stout_default_choice(f->prec);
  if (!tune_enabled()) return LQ_OK;
  if (tune_get("stout", f->prec, f->geom.dims, dirs, out)) return LQ_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone) return LQ_OK;  // never tune inside a capture
  lq_status st = stout_autotune(f, rho, dirs, reproject, s, out);
  if (st != LQ_OK) return st;
  tune_put("stout", f->prec, f->geom.dims, dirs, *out);
  return LQ_OK;
}

// ---- CUDA-graph cache for the n-step sequence ------------------------------
struct GraphKey {
  void* links;
  int dims[4];
  int prec, n, reproject, block, nsite, variant, device;
  unsigned dirs;
  double rho;
  bool operator<(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) < 0; }
};
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  void* work = nullptr;
  void* wfield = nullptr;   // two-link products (variant 3)
  unsigned long long used = 0;
};
// At most kMaxGraphs recorded sequences are kept (each holds a links-sized
// workspace); the least recently launched one is dropped first.
constexpr size_t kMaxGraphs = 8;
static std::mutex g_graph_mu;
static unsigned long long g_graph_tick = 0;
static std::map<GraphKey, GraphEntry>& graph_cache() {
  static std::map<GraphKey, GraphEntry> m;
  return m;
}
static void free_graph_entry(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.work) cudaFree(e.work);
  if (e.wfield) cudaFree(e.wfield);
  e = GraphEntry();
}
static void release_graphs() {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto& kv : graph_cache()) free_graph_entry(kv.second);
  graph_cache().clear();
}

static lq_status run_graph(lq_field* f, double rho, int n, unsigned dirs, int reproject, const TuneChoice& tc,
                           cudaStream_t s) {
  register_cache_release(release_graphs);
  GraphKey k;
  std::memset(&k, 0, sizeof(k));
  k.links = f->ptr;
  for (int i = 0; i < 4; ++i) k.dims[i] = f->geom.dims[i];
  k.prec = f->prec;
  k.n = n;
  k.reproject = reproject;
  k.block = tc.block;
  k.nsite = tc.nsite;
  k.variant = tc.variant;
  k.device = current_device();
  k.dirs = dirs;
  k.rho = rho;
  std::lock_guard<std::mutex> lk(g_graph_mu);
  const unsigned long long now = ++g_graph_tick;
  auto it = graph_cache().find(k);
  if (it == graph_cache().end()) {
    while (graph_cache().size() >= kMaxGraphs) {   // cudaFree waits for launches still using the entry
      auto old = graph_cache().begin();
      for (auto j = graph_cache().begin(); j != graph_cache().end(); ++j)
        if (j->second.used < old->second.used) old = j;
      free_graph_entry(old->second);
      graph_cache().erase(old);
    }
    GraphEntry e;
    lq_status st = cuda_check(cudaMalloc(&e.work, f->bytes), "stout graph workspace");
    if (st != LQ_OK) return st;
    if (tc.variant == 3) {
      st = cuda_check(cudaMalloc(&e.wfield, wfield_bytes(f->geom, f->prec, dirs)), "stout graph two-link products");
      if (st != LQ_OK) {
        cudaFree(e.work);
        return st;
      }
    }
    cudaStream_t cap;
    st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stout graph stream");
    if (st != LQ_OK) {
      cudaFree(e.work);
      return st;
    }
    cudaGraph_t graph = nullptr;
    st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "stout graph capture");
    if (st == LQ_OK) {
      lq_status st_run = stout_run_steps(f->ptr, e.work, f->geom, f->prec, rho, n, dirs, reproject, tc, cap, e.wfield);
      lq_status st_end = cuda_check(cudaStreamEndCapture(cap, &graph), "stout graph end capture");
      st = st_run != LQ_OK ? st_run : st_end;
    }
    if (st == LQ_OK) st = cuda_check(cudaGraphInstantiate(&e.exec, graph, 0), "stout graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st != LQ_OK) {
      cudaFree(e.work);
      if (e.wfield) cudaFree(e.wfield);
      return st;
    }
    it = graph_cache().emplace(k, e).first;
  }
  it->second.used = now;
  return cuda_check(cudaGraphLaunch(it->second.exec, s), "stout graph launch");
}

}  // namespace lq

namespace lq {

// exp(iQ) per site of a COLOR_MATRIX field (the stout step's exponential alone).
template <typename R>
__global__ void k_expiq(const typename vec2<R>::type* __restrict__ Q, typename vec2<R>::type* __restrict__ E,
                        long long V) {
  const long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= V) return;
  const M3<R> m = ld_m3<R>(Q + sl, V);
  QH<R> q;
  q.d0 = m.e[0].re;
  q.d1 = m.e[4].re;
  q.d2 = m.e[8].re;
  q.o01 = m.e[1];
  q.o02 = m.e[2];
  q.o12 = m.e[5];
  // any input: its trace removed in FP64 before the coefficients (which take
  // the diagonal as traceless up to rounding)
  const double d0 = to_f64(q.d0), d1 = to_f64(q.d1), d2 = to_f64(q.d2);
  const double tq = (d0 + d1 + d2) * (1.0 / 3.0);
  const CHCoef f = ch_coefficients<sizeof(R) == 4 ? 1 : 2>(d0 - tq, d1 - tq, d2 - tq,
                                                           mkc(to_f64(q.o01.re), to_f64(q.o01.im)),
                                                           mkc(to_f64(q.o02.re), to_f64(q.o02.im)),
                                                           mkc(to_f64(q.o12.re), to_f64(q.o12.im)));
  // the coefficients belong to the traceless part of Q: assemble with it
  const R t = (q.d0 + q.d1 + q.d2) * R(1.0 / 3.0);
  q.d0 -= t;
  q.d1 -= t;
  q.d2 -= t;
  const M3<R> e = expiq_assemble(q, q_square(q), mkc<R>(from_f64<R>(f.f0.re), from_f64<R>(f.f0.im)),
                                 mkc<R>(from_f64<R>(f.f1.re), from_f64<R>(f.f1.im)),
                                 mkc<R>(from_f64<R>(f.f2.re), from_f64<R>(f.f2.im)));
  st_m3<R>(E + sl, V, e);
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_expiq(lq_field* out, const lq_field* q, void* stream) {
  clear_error();
  if (!out || !q) {
    set_error("lq_expiq: NULL field");
    return LQ_ERR_ARG;
  }
  if (out->kind != LQ_COLOR_MATRIX || q->kind != LQ_COLOR_MATRIX || out->prec != q->prec ||
      !same_geom(out->geom, q->geom)) {
    set_error("lq_expiq: out and q must be COLOR_MATRIX fields of one geometry and precision");
    return LQ_ERR_GEOM;
  }
  if (out->ptr == q->ptr) {
    set_error("lq_expiq: out must not alias q");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  const long long V = q->geom.volume;
  const unsigned grid = (unsigned)((V + 127) / 128);
  if (q->prec == LQ_F64)
    k_expiq<double><<<grid, 128, 0, s>>>((const double2*)q->ptr, (double2*)out->ptr, V);
  else
    k_expiq<float><<<grid, 128, 0, s>>>((const float2*)q->ptr, (float2*)out->ptr, V);
  return launch_check("lq_expiq");
}

extern "C" lq_status lq_stout_smear(lq_field* links, double rho, int n_steps, unsigned dirs_mask,
                                    const lq_stout_opts* opts, void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_stout_smear");
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_stout_smear")) != LQ_OK) return st;
  if (!(rho >= 0.0) || rho > 1e6) {
    set_error("lq_stout_smear: rho must be finite and >= 0");
    return LQ_ERR_ARG;
  }
  if (n_steps < 0) {
    set_error("lq_stout_smear: n_steps must be >= 0");
    return LQ_ERR_ARG;
  }
  const lq_stout_opts* o = (opts && opts->struct_size >= (int)sizeof(lq_stout_opts)) ? opts : nullptr;
  if (opts && !o && opts->struct_size != 0) {
    set_error("lq_stout_smear: opts->struct_size %d < sizeof(lq_stout_opts)", opts->struct_size);
    return LQ_ERR_ARG;
  }
  if (o && (o->variant < 0 || o->variant > 3)) {
    set_error("lq_stout_smear: variant %d is not available (0 tuned, 1 global, 2 shared memory, "
              "3 two-link products)", o->variant);
    return LQ_ERR_UNSUPPORTED;
  }
  if (o && o->variant == 2 && links->prec != LQ_F32) {
    set_error("lq_stout_smear: the shared-memory variant is built for FP32 links only");
    return LQ_ERR_UNSUPPORTED;
  }
  if (o && o->block > 0 && o->variant != 2 && (o->block % 32 != 0 || o->block > 256)) {
    set_error("lq_stout_smear: block %d must be a multiple of 32 in [32, 256]", o->block);
    return LQ_ERR_ARG;
  }
  if (n_steps == 0) return LQ_OK;
  cudaStream_t s = as_stream(stream);
  const int reproject = (o && o->reproject >= 0) ? o->reproject : (links->prec == LQ_F32 ? 1 : 0);
  TuneChoice tc;
  if ((st = stout_choose(links, rho, dirs_mask, reproject, o, s, &tc)) != LQ_OK) return st;
  if (o && o->use_graph) return run_graph(links, rho, n_steps, dirs_mask, reproject, tc, s);
  void* work = nullptr;
  bool own = false;
  if (o && o->work) {
    if (o->work_bytes < links->bytes || (((uintptr_t)o->work) & 15u)) {
      set_error("lq_stout_smear: opts->work must be 16-byte aligned and hold %zu bytes", links->bytes);
      return LQ_ERR_ARG;
    }
    work = o->work;
  } else {
    if ((st = scratch_alloc(&work, links->bytes, s, "lq_stout_smear workspace")) != LQ_OK) return st;
    own = true;
  }
  st = stout_run_steps(links->ptr, work, links->geom, links->prec, rho, n_steps, dirs_mask, reproject, tc, s);
  if (own) scratch_free(work, s);
  return st;
}

extern "C" lq_status lq_stout_step_range(const lq_field* in, lq_field* out, double rho, unsigned dirs_mask,
                                         long long s_begin, long long s_end, const lq_stout_opts* opts,
                                         void* stream) {
  clear_error();
  lq_status st = check_links(in, "lq_stout_step_range");
  if (st != LQ_OK) return st;
  if ((st = check_links(out, "lq_stout_step_range")) != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_stout_step_range")) != LQ_OK) return st;
  if (out->prec != in->prec || !same_geom(out->geom, in->geom)) {
    set_error("lq_stout_step_range: in and out must share geometry and precision");
    return LQ_ERR_GEOM;
  }
  if (out->ptr == in->ptr) {
    set_error("lq_stout_step_range: out must not alias in");
    return LQ_ERR_ARG;
  }
  if (!(rho >= 0.0) || rho > 1e6 || s_begin < 0 || s_end < s_begin || s_end > in->geom.volume) {
    set_error("lq_stout_step_range: need finite rho >= 0 and 0 <= s_begin <= s_end <= volume");
    return LQ_ERR_ARG;
  }
  if (s_end == s_begin) return LQ_OK;
  const lq_stout_opts* o = (opts && opts->struct_size >= (int)sizeof(lq_stout_opts)) ? opts : nullptr;
  const int reproject = (o && o->reproject >= 0) ? o->reproject : (in->prec == LQ_F32 ? 1 : 0);
  TuneChoice tc = stout_default_choice(in->prec);
  if (o && o->block > 0) {
    if (o->block % 32 != 0 || o->block > 256) {
      set_error("lq_stout_step_range: block must be a multiple of 32 in [32, 256]");
      return LQ_ERR_ARG;
    }
    tc.block = o->block;
    tc.nsite = o->sites_per_thread > 0 ? o->sites_per_thread : 1;
  } else if (tune_enabled()) {
    tune_get("stout", in->prec, in->geom.dims, dirs_mask, &tc);
  }
  return stout_step_range(in->ptr, out->ptr, in->geom, in->prec, rho, dirs_mask, reproject, tc, s_begin, s_end,
                          as_stream(stream));
}

extern "C" lq_status lq_stout_ch_stats(const lq_field* links, double rho, int n_steps, unsigned dirs_mask,
                                       long long* counts, void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_stout_ch_stats");
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_stout_ch_stats")) != LQ_OK) return st;
  if (!(rho >= 0.0) || rho > 1e6 || n_steps < 0 || !counts) {
    set_error("lq_stout_ch_stats: need finite rho >= 0, n_steps >= 0 and a counts array");
    return LQ_ERR_ARG;
  }
  for (int i = 0; i < 3; ++i) counts[i] = 0;
  if (n_steps == 0) return LQ_OK;
  cudaStream_t s = as_stream(stream);
  void* buf[2] = {nullptr, nullptr};
  void* dstats = nullptr;
  for (int i = 0; i < 2 && st == LQ_OK; ++i) {
    st = scratch_alloc(&buf[i], links->bytes, s, "lq_stout_ch_stats fields");
    // links outside dirs are read by the staples and never written: both copies hold them
    if (st == LQ_OK)
      st = cuda_check(cudaMemcpyAsync(buf[i], links->ptr, links->bytes, cudaMemcpyDeviceToDevice, s),
                      "lq_stout_ch_stats copy");
  }
  if (st == LQ_OK) st = scratch_alloc(&dstats, 3 * sizeof(unsigned long long), s, "lq_stout_ch_stats counters");
  if (st == LQ_OK)
    st = cuda_check(cudaMemsetAsync(dstats, 0, 3 * sizeof(unsigned long long), s), "lq_stout_ch_stats counters");
  const GeomArgs g = geom_args(links->geom);
  int nd = 0;
  const MuList ml = mu_list(dirs_mask, &nd);
  const int block = 128;
  const dim3 grid((unsigned)(((g.V + block - 1) / block) * nd));
  unsigned long long* ds = (unsigned long long*)dstats;
  for (int k = 0; k < n_steps && st == LQ_OK; ++k) {
    const void* in = buf[k % 2];
    void* out = buf[(k + 1) % 2];
    if (links->prec == LQ_F64)
      k_stout_global_f64<false, true><<<grid, block, 0, s>>>((const double2*)in, (double2*)out, g, rho,
                                                                 dirs_mask, 1, nd, ml, ds, 0, g.V);
    else
      k_stout_global_f32<true, true><<<grid, block, 0, s>>>((const float2*)in, (float2*)out, g, (float)rho,
                                                               dirs_mask, 1, nd, ml, ds, 0, g.V);
    st = launch_check("lq_stout_ch_stats step");
  }
  unsigned long long h[3] = {0, 0, 0};
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpyAsync(h, dstats, sizeof(h), cudaMemcpyDeviceToHost, s), "lq_stout_ch_stats read");
  if (st == LQ_OK) st = cuda_check(cudaStreamSynchronize(s), "lq_stout_ch_stats sync");
  for (int i = 0; i < 2; ++i)
    if (buf[i]) scratch_free(buf[i], s);
  if (dstats) scratch_free(dstats, s);
  if (st == LQ_OK)
    for (int i = 0; i < 3; ++i) counts[i] = (long long)h[i];
  return st;
}
