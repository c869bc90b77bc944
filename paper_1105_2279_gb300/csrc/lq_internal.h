// Internal host-side definitions shared by the liblqcd translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/lqcd.h"
#include "geom.cuh"

struct lq_geom {
  int dims[4];
  long long volume;
};

struct lq_field {
  lq_geom geom;      // copied, so a field outlives its geometry handle
  int kind;
  int prec;
  void* ptr;
  size_t bytes;
  bool owned;
};

namespace lq {

// Thread-local last error message.
void set_error(const char* fmt, ...);
void clear_error();

inline int ndir_of(int kind) { return kind == LQ_LINKS ? 4 : 1; }
inline int ncomp_of(int kind) {
  switch (kind) {
    case LQ_LINKS:
    case LQ_COLOR_MATRIX: return 9;
    case LQ_COLOR_VECTOR: return 3;
    case LQ_FERMION: return 12;
    default: return 1;
  }
}
inline size_t elem_bytes(int kind, int prec) {
  size_t r = prec == LQ_F64 ? 8 : 4;
  return kind == LQ_REAL ? r : 2 * r;
}
inline bool valid_kind(int k) { return k >= LQ_LINKS && k <= LQ_FERMION; }
inline bool valid_prec(int p) { return p == LQ_F32 || p == LQ_F64; }
inline size_t field_bytes(const lq_geom& g, int kind, int prec) {
  return (size_t)g.volume * ndir_of(kind) * ncomp_of(kind) * elem_bytes(kind, prec);
}
inline bool same_geom(const lq_geom& a, const lq_geom& b) {
  return a.dims[0] == b.dims[0] && a.dims[1] == b.dims[1] && a.dims[2] == b.dims[2] &&
         a.dims[3] == b.dims[3];
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Returns LQ_ERR_CUDA (with message) if e != cudaSuccess.
lq_status cuda_check(cudaError_t e, const char* what);
// Checks the launch just issued.
lq_status launch_check(const char* what);

int device_sm_count();
int current_device();

// Stream-ordered scratch allocation that reports OOM as LQ_ERR_OOM.
lq_status scratch_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
void scratch_free(void* p, cudaStream_t s);

inline GeomArgs geom_args(const lq_geom& g) {
  GeomArgs a;
  int st = 1;
  for (int i = 0; i < 4; ++i) {
    a.L[i] = g.dims[i];
    a.stride[i] = st;
    st *= g.dims[i];
  }
  a.V = (int)g.volume;
  return a;
}

// Validation helpers (set the error message and return the status).
lq_status check_links(const lq_field* f, const char* who);
lq_status check_dirs(unsigned mask, const char* who);

// Autotuner (tune.cu).
struct TuneChoice {
  int block;
  int nsite;
  int variant;
};
bool tune_enabled();
bool tune_get(const char* kernel, int prec, const int dims[4], unsigned dirs, TuneChoice* out);
void tune_put(const char* kernel, int prec, const int dims[4], unsigned dirs, const TuneChoice& c);

// Stout internals shared with the backward and batch translation units.
// wbuf: two-link product buffer for variant 3 (NULL: allocated per call when needed)
lq_status stout_run_steps(void* links, void* work, const lq_geom& g, int prec, double rho,
                          int n_steps, unsigned dirs, int reproject, const TuneChoice& tc,
                          cudaStream_t s, void* wbuf = nullptr);
TuneChoice stout_default_choice(int prec);
// n APE steps in place on the link field `links` (bytes long), with `work` a
// scratch field of the same size; the arithmetic of lq_ape_smear.
lq_status ape_run_steps(void* links, void* work, const lq_geom& g, int prec, size_t bytes, double alpha,
                        int n_steps, unsigned dirs, cudaStream_t s);
// One APE step from `in` to `out` (distinct fields); directions outside dirs
// are not written.
lq_status ape_step(const void* in, void* out, const lq_geom& g, int prec, double alpha, unsigned dirs,
                   cudaStream_t s);
// n HYP steps in place; scratch holds 24 colour-matrix planes (bytes / 4 each).
lq_status hyp_run_steps(void* links, void* work, void* scratch, const lq_geom& g, int prec, size_t bytes,
                        double a1, double a2, double a3, int n_steps, cudaStream_t s);
// Gradient through one HYP step: Gout = G at U^(k) from Gp = G at U^(k+1);
// scratch holds kHypBwdPlanes colour-matrix planes.
constexpr int kHypBwdPlanes = 64;
lq_status hyp_backward_step(const void* Uk, const void* Gp, void* Gout, void* scratch, const lq_geom& g, int prec,
                            size_t bytes, double a1, double a2, double a3, cudaStream_t s);
// One stout step over the sites [s_begin, s_end) only (global-load kernel).
lq_status stout_step_range(const void* in, void* out, const lq_geom& g, int prec, double rho, unsigned dirs,
                           int reproject, const TuneChoice& tc, long long s_begin, long long s_end,
                           cudaStream_t s);
// Independent site ranges, each with its own input and output field, in one
// launch per kMaxSegs ranges (the same per-link arithmetic as lq_stout_smear).
constexpr int kMaxSegs = 8;
struct StepSegment {
  const void* in;
  void* out;
  long long s_begin, s_end;
};
lq_status stout_step_segments(const StepSegment* seg, int nseg, const lq_geom& g, int prec, double rho,
                              unsigned dirs, int reproject, const TuneChoice& tc, cudaStream_t s);
// AoS <-> SoA transpose of the sites [s_begin, s_end) of a field of this kind,
// between a whole-lattice AoS buffer and a whole-lattice SoA buffer.
lq_status transpose_range(const void* src, void* dst, const lq_geom& g, int kind, int prec, bool to_soa,
                          long long s_begin, long long s_end, cudaStream_t s);
// The device address of page-locked host memory (the GPU reads and writes it
// over the host link), or NULL for memory the GPU cannot address directly.
void* host_device_view(const void* p);
lq_status stout_choose(const lq_field* f, double rho, unsigned dirs, int reproject,
                       const lq_stout_opts* o, cudaStream_t s, TuneChoice* out);

// Reductions shared by several entry points.
lq_status plaquette_sums(const lq_field* links, double out_planes[2], cudaStream_t s);
lq_status plaquette_sums_device(const lq_field* links, double* dev_totals, cudaStream_t s);
void plaquette_from_sums(const double sums[2], long long volume, double out[3]);

// Registered cleanup callbacks for lq_free_all.
void register_cache_release(void (*fn)());

}  // namespace lq
