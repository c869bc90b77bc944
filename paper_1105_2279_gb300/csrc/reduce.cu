// Global reductions with FP64 accumulation: plaquette, Wilson action, sum and
// trace-sum of a field.  Per-site products run in the field precision; the
// sums go through reduce.cuh's deterministic two-pass tree.
#include "lq_internal.h"
#include "reduce.cuh"
#include "stout_core.cuh"

namespace lq {

// Re tr P_{mu nu}(x) = Re tr[(U_mu(x) U_nu(x+mu)) (U_nu(x) U_mu(x+nu))^dag],
// summed over the spatial planes (nu < 3) and the temporal planes (nu = 3).
// Sites [s0, s1) (the whole lattice, or the slab a rank owns).  FP32 links:
// held to 128 registers, two 256-thread blocks per SM (at the 130 it would
// take unbounded, one block of 8 warps per SM left the loads' latency bare).
template <typename R>
__global__ void __launch_bounds__(kReduceThreads, sizeof(R) == 4 ? 2 : 1) k_plaquette(const typename vec2<R>::type* __restrict__ U,
                                                              GeomArgs g, long long s0, long long s1,
                                                              double* __restrict__ parts) {
  double v[2] = {0.0, 0.0};
  const long long V = g.V;
  for (long long sl = s0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < s1;
       sl += (long long)gridDim.x * blockDim.x) {
    const int s = (int)sl;
    int c[4];
    site_coords(g, s, c);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
      const int s_pmu = nb_fwd(g, s, c[mu], mu);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int s_pnu = nb_fwd(g, s, c[nu], nu);
        const M3<R> a = mul_nn(ld_link<R>(U, V, mu, s), ld_link<R>(U, V, nu, s_pmu));
        const M3<R> b = mul_nn(ld_link<R>(U, V, nu, s), ld_link<R>(U, V, mu, s_pnu));
        v[nu == 3 ? 1 : 0] += (double)retr_nd(a, b);
      }
    }
  }
  block_sum_store<2>(v, parts + 2 * blockIdx.x);
}

// Sum over all elements (re, im) of a field with element type E.
__device__ __forceinline__ void elem_acc2(float2 e, double (&v)[2]) {
  v[0] += e.x;
  v[1] += e.y;
}
__device__ __forceinline__ void elem_acc2(double2 e, double (&v)[2]) {
  v[0] += e.x;
  v[1] += e.y;
}
__device__ __forceinline__ void elem_acc2(float e, double (&v)[2]) { v[0] += e; }
__device__ __forceinline__ void elem_acc2(double e, double (&v)[2]) { v[0] += e; }

template <typename E>
__global__ void __launch_bounds__(kReduceThreads) k_sum(const E* __restrict__ f, long long n, double* parts) {
  double v[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    elem_acc2(__ldg(f + i), v);
  block_sum_store<2>(v, parts + 2 * blockIdx.x);
}

// sum_x tr M(x) over ndir matrix fields of V sites each.
template <typename E>
__global__ void __launch_bounds__(kReduceThreads) k_trace(const E* __restrict__ f, long long V, int ndir,
                                                          double* parts) {
  double v[2] = {0.0, 0.0};
  const long long n = V * ndir;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long d = i / V, s = i - d * V;
    const E* p = f + d * 9 * V + s;
    elem_acc2(__ldg(p), v);
    elem_acc2(__ldg(p + 4 * V), v);
    elem_acc2(__ldg(p + 8 * V), v);
  }
  block_sum_store<2>(v, parts + 2 * blockIdx.x);
}

// Runs `launch(parts)` (which writes `grid` partial pairs), reduces them and
// copies the two totals to host.  Synchronises s.
template <typename F>
static lq_status reduce_two(int grid, cudaStream_t s, double out[2], const char* who, F launch) {
  double* scratch = nullptr;
  lq_status st = scratch_alloc((void**)&scratch, sizeof(double) * 2 * (grid + 1), s, who);
  if (st != LQ_OK) return st;
  launch(scratch);
  st = launch_check(who);
  if (st == LQ_OK) {
    k_reduce_partials<2><<<1, kReduceThreads, 0, s>>>(scratch, grid, scratch + 2 * grid);
    st = launch_check(who);
  }
  double host[2] = {0.0, 0.0};
  if (st == LQ_OK) st = cuda_check(cudaMemcpyAsync(host, scratch + 2 * grid, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), who);
  scratch_free(scratch, s);
  lq_status st2 = cuda_check(cudaStreamSynchronize(s), who);
  if (st == LQ_OK) st = st2;
  if (st == LQ_OK) {
    out[0] = host[0];
    out[1] = host[1];
  }
  return st;
}

static lq_status plaquette_sums_range(const lq_field* links, long long s0, long long s1, double out_planes[2],
                                      cudaStream_t s) {
  const GeomArgs g = geom_args(links->geom);
  const int grid = reduce_grid(s1 - s0);
  return reduce_two(grid, s, out_planes, "lq_plaquette", [&](double* parts) {
    if (links->prec == LQ_F64)
      k_plaquette<double><<<grid, kReduceThreads, 0, s>>>((const double2*)links->ptr, g, s0, s1, parts);
    else
      k_plaquette<float><<<grid, kReduceThreads, 0, s>>>((const float2*)links->ptr, g, s0, s1, parts);
  });
}

lq_status plaquette_sums(const lq_field* links, double out_planes[2], cudaStream_t s) {
  return plaquette_sums_range(links, 0, links->geom.volume, out_planes, s);
}

// The two plane sums of the whole field into dev_totals[0..1] on the device,
// stream-ordered on s (the same kernels and order as plaquette_sums, without
// the read-back): a caller that reads them back on another stream.
lq_status plaquette_sums_device(const lq_field* links, double* dev_totals, cudaStream_t s) {
  const GeomArgs g = geom_args(links->geom);
  const long long V = links->geom.volume;
  const int grid = reduce_grid(V);
  double* parts = nullptr;
  lq_status st = scratch_alloc((void**)&parts, sizeof(double) * 2 * grid, s, "lq_plaquette");
  if (st != LQ_OK) return st;
  if (links->prec == LQ_F64)
    k_plaquette<double><<<grid, kReduceThreads, 0, s>>>((const double2*)links->ptr, g, 0, V, parts);
  else
    k_plaquette<float><<<grid, kReduceThreads, 0, s>>>((const float2*)links->ptr, g, 0, V, parts);
  st = launch_check("lq_plaquette");
  if (st == LQ_OK) {
    k_reduce_partials<2><<<1, kReduceThreads, 0, s>>>(parts, grid, dev_totals);
    st = launch_check("lq_plaquette");
  }
  scratch_free(parts, s);
  return st;
}

void plaquette_from_sums(const double sums[2], long long volume, double out[3]) {
  const double V = (double)volume;
  out[0] = (sums[0] + sums[1]) / (18.0 * V);
  out[1] = sums[0] / (9.0 * V);
  out[2] = sums[1] / (9.0 * V);
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_plaquette(const lq_field* links, double out[3], void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_plaquette");
  if (st != LQ_OK) return st;
  if (!out) {
    set_error("lq_plaquette: NULL output");
    return LQ_ERR_ARG;
  }
  double sums[2];
  st = plaquette_sums(links, sums, as_stream(stream));
  if (st != LQ_OK) return st;
  plaquette_from_sums(sums, links->geom.volume, out);
  return LQ_OK;
}

extern "C" lq_status lq_plaquette_sums(const lq_field* links, long long s_begin, long long s_end, double out[2],
                                       void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_plaquette_sums");
  if (st != LQ_OK) return st;
  if (!out || s_begin < 0 || s_end < s_begin || s_end > links->geom.volume) {
    set_error("lq_plaquette_sums: need an output and 0 <= s_begin <= s_end <= volume");
    return LQ_ERR_ARG;
  }
  if (s_end == s_begin) {
    out[0] = out[1] = 0.0;
    return LQ_OK;
  }
  return plaquette_sums_range(links, s_begin, s_end, out, as_stream(stream));
}

extern "C" lq_status lq_wilson_action(const lq_field* links, double beta, double* out, void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_wilson_action");
  if (st != LQ_OK) return st;
  if (!out) {
    set_error("lq_wilson_action: NULL output");
    return LQ_ERR_ARG;
  }
  double sums[2];
  st = plaquette_sums(links, sums, as_stream(stream));
  if (st != LQ_OK) return st;
  const double V = (double)links->geom.volume;
  *out = beta * (6.0 * V - (sums[0] + sums[1]) / 3.0);
  return LQ_OK;
}

extern "C" lq_status lq_reduce_sum(const lq_field* f, double out[2], void* stream) {
  clear_error();
  if (!f || !out) {
    set_error("lq_reduce_sum: NULL argument");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  const long long n = f->geom.volume * ndir_of(f->kind) * ncomp_of(f->kind);
  const int grid = reduce_grid(n);
  const size_t eb = elem_bytes(f->kind, f->prec);
  return reduce_two(grid, s, out, "lq_reduce_sum", [&](double* parts) {
    if (f->kind == LQ_REAL) {
      if (f->prec == LQ_F64)
        k_sum<double><<<grid, kReduceThreads, 0, s>>>((const double*)f->ptr, n, parts);
      else
        k_sum<float><<<grid, kReduceThreads, 0, s>>>((const float*)f->ptr, n, parts);
    } else if (eb == 16) {
      k_sum<double2><<<grid, kReduceThreads, 0, s>>>((const double2*)f->ptr, n, parts);
    } else {
      k_sum<float2><<<grid, kReduceThreads, 0, s>>>((const float2*)f->ptr, n, parts);
    }
  });
}

extern "C" lq_status lq_reduce_trace(const lq_field* f, double out[2], void* stream) {
  clear_error();
  if (!f || !out) {
    set_error("lq_reduce_trace: NULL argument");
    return LQ_ERR_ARG;
  }
  if (f->kind != LQ_LINKS && f->kind != LQ_COLOR_MATRIX) {
    set_error("lq_reduce_trace: field kind %d is not a matrix field", f->kind);
    return LQ_ERR_GEOM;
  }
  cudaStream_t s = as_stream(stream);
  const long long V = f->geom.volume;
  const int ndir = ndir_of(f->kind);
  const int grid = reduce_grid(V * ndir);
  return reduce_two(grid, s, out, "lq_reduce_trace", [&](double* parts) {
    if (f->prec == LQ_F64)
      k_trace<double2><<<grid, kReduceThreads, 0, s>>>((const double2*)f->ptr, V, ndir, parts);
    else
      k_trace<float2><<<grid, kReduceThreads, 0, s>>>((const float2*)f->ptr, V, ndir, parts);
  });
}
