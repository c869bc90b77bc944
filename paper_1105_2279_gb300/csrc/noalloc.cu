// lq_stout_smear_noalloc: stout smearing that allocates no device memory.
//
// lq_stout_smear needs a second links field as its double buffer and gets it
// from cudaMallocAsync.  Some callers cannot let a library allocate: code
// running where every byte of device memory is already reserved by the host
// application's own allocator (a framework that owns the pool), plug-ins whose
// host forbids device allocations, and latency-critical paths that must not
// risk the synchronisation or failure an allocation can bring.  For them this
// entry point takes its double buffer from a file-scope __device__ array of
// LQ_NOALLOC_WORK_BYTES (32 MiB), which every GPU that loads the library holds
// until the process exits.
#include <mutex>

#include "lq_internal.h"

namespace lq {

static __device__ __align__(256) unsigned char g_noalloc_work[LQ_NOALLOC_WORK_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_work on the current device, looked up once per
// device (host code only sees a host-side stand-in for the symbol).
static lq_status noalloc_workspace(void** out) {
  const int dev = current_device();
  if (dev < 0 || dev >= 64) {
    set_error("lq_stout_smear_noalloc: device ordinal %d out of range", dev);
    return LQ_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    lq_status st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_work), "lq_stout_smear_noalloc set-up");
    if (st != LQ_OK) return st;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_stout_smear_noalloc(lq_field* links, double rho, int n_steps, unsigned dirs_mask,
                                            void* stream) {
  clear_error();
  lq_status st = check_links(links, "lq_stout_smear_noalloc");
  if (st != LQ_OK) return st;
  if ((st = check_dirs(dirs_mask, "lq_stout_smear_noalloc")) != LQ_OK) return st;
  if (!(rho >= 0.0) || rho > 1e6 || n_steps < 0) {
    set_error("lq_stout_smear_noalloc: rho must be finite >= 0 and n_steps >= 0");
    return LQ_ERR_ARG;
  }
  if (links->bytes > (size_t)LQ_NOALLOC_WORK_BYTES) {
    set_error("lq_stout_smear_noalloc: the links field needs a %zu-byte double buffer, more than the %zu bytes "
              "of the built-in workspace; use lq_stout_smear",
              links->bytes, (size_t)LQ_NOALLOC_WORK_BYTES);
    return LQ_ERR_ARG;
  }
  if (n_steps == 0) return LQ_OK;
  void* work = nullptr;
  if ((st = noalloc_workspace(&work)) != LQ_OK) return st;
  // tuned launch shape if one is cached; never runs the tuner (it allocates)
  TuneChoice tc = stout_default_choice(links->prec);
  if (tune_enabled()) tune_get("stout", links->prec, links->geom.dims, dirs_mask, &tc);
  if (tc.variant == 3) tc = stout_default_choice(links->prec);   // variant 3 needs a product buffer
  const int reproject = links->prec == LQ_F32 ? 1 : 0;
  return stout_run_steps(links->ptr, work, links->geom, links->prec, rho, n_steps, dirs_mask, reproject, tc,
                         as_stream(stream));
}
