// Geometry, field handles, host<->device transfers, error reporting and the
// device-storage release of liblqcd (device residency API of Winter,
// "Accelerating QDP++ using GPUs", Sec. 5; coalesced layout, Sec. 8).
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lq_internal.h"

namespace lq {

static thread_local char g_err[512] = {0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

lq_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LQ_OK;
  set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return LQ_ERR_OOM;
  return LQ_ERR_CUDA;
}

lq_status launch_check(const char* what) { return cuda_check(cudaGetLastError(), what); }

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int device_sm_count() {
  static int cached[64] = {0};
  int d = current_device();
  if (d < 0 || d >= 64) return 152;
  if (!cached[d]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 152;
    cached[d] = n;
  }
  return cached[d];
}

lq_status scratch_alloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("%s: could not allocate %zu bytes of device scratch (%s)", what, bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LQ_ERR_OOM : LQ_ERR_CUDA;
  }
  return LQ_OK;
}

void scratch_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

lq_status check_links(const lq_field* f, const char* who) {
  if (!f) {
    set_error("%s: links field is NULL", who);
    return LQ_ERR_ARG;
  }
  if (f->kind != LQ_LINKS) {
    set_error("%s: field kind %d is not LQ_LINKS", who, f->kind);
    return LQ_ERR_GEOM;
  }
  return LQ_OK;
}

lq_status check_dirs(unsigned mask, const char* who) {
  if (mask == 0 || mask > 15u) {
    set_error("%s: dirs_mask %u must be in [1, 15]", who, mask);
    return LQ_ERR_ARG;
  }
  return LQ_OK;
}

static std::mutex g_release_mu;
static std::vector<void (*)()>& release_list() {
  static std::vector<void (*)()> v;
  return v;
}
void register_cache_release(void (*fn)()) {
  std::lock_guard<std::mutex> lk(g_release_mu);
  for (auto f : release_list())
    if (f == fn) return;
  release_list().push_back(fn);
}

// ---- AoS <-> SoA transposes ------------------------------------------------
// One thread per (site, element-in-site): reads of a warp are contiguous in
// the AoS buffer, writes go to per-component planes.
template <typename E>
__global__ void aos_to_soa(const E* __restrict__ aos, E* __restrict__ soa, long long V, int per_site) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = V * per_site;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long s = i / per_site;
    int c = (int)(i - s * per_site);
    soa[(long long)c * V + s] = aos[i];
  }
}
template <typename E>
__global__ void soa_to_aos(const E* __restrict__ soa, E* __restrict__ aos, long long V, int per_site) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = V * per_site;
  for (; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long s = i / per_site;
    int c = (int)(i - s * per_site);
    aos[i] = soa[(long long)c * V + s];
  }
}

static lq_status transpose(const void* src, void* dst, const lq_field* f, bool to_soa, cudaStream_t s) {
  const long long V = f->geom.volume;
  const int per_site = ndir_of(f->kind) * ncomp_of(f->kind);
  const size_t eb = elem_bytes(f->kind, f->prec);
  const long long n = V * per_site;
  int blocks = (int)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 16);
  if (blocks < 1) blocks = 1;
#define LQ_T(E)                                                                                   \
  if (to_soa)                                                                                     \
    aos_to_soa<E><<<blocks, 256, 0, s>>>((const E*)src, (E*)dst, V, per_site);                   \
  else                                                                                            \
    soa_to_aos<E><<<blocks, 256, 0, s>>>((const E*)src, (E*)dst, V, per_site);
  if (eb == 4) {
    LQ_T(float)
  } else if (eb == 8) {
    LQ_T(float2)
  } else {
    LQ_T(double2)
  }
#undef LQ_T
  return launch_check(to_soa ? "aos_to_soa" : "soa_to_aos");
}

}  // namespace lq

using namespace lq;

extern "C" {

const char* lq_last_error(void) { return g_err; }

int lq_abi_version(void) { return 1; }

lq_status lq_geom_create(const int dims[4], lq_geom** out) {
  clear_error();
  if (!dims || !out) {
    set_error("lq_geom_create: NULL argument");
    return LQ_ERR_ARG;
  }
  long long v = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 1) {
      set_error("lq_geom_create: dims[%d] = %d must be >= 1", i, dims[i]);
      return LQ_ERR_ARG;
    }
    v *= dims[i];
    if (v >= (1LL << 31)) {
      set_error("lq_geom_create: volume must be < 2^31 sites");
      return LQ_ERR_ARG;
    }
  }
  lq_geom* g = new (std::nothrow) lq_geom;
  if (!g) {
    set_error("lq_geom_create: host allocation failed");
    return LQ_ERR_OOM;
  }
  for (int i = 0; i < 4; ++i) g->dims[i] = dims[i];
  g->volume = v;
  *out = g;
  return LQ_OK;
}

lq_status lq_geom_destroy(lq_geom* g) {
  clear_error();
  delete g;
  return LQ_OK;
}

lq_status lq_geom_info(const lq_geom* g, int dims_out[4], long long* volume_out) {
  clear_error();
  if (!g) {
    set_error("lq_geom_info: NULL geometry");
    return LQ_ERR_ARG;
  }
  if (dims_out)
    for (int i = 0; i < 4; ++i) dims_out[i] = g->dims[i];
  if (volume_out) *volume_out = g->volume;
  return LQ_OK;
}

lq_status lq_field_bytes(const lq_geom* g, int kind, int prec, size_t* bytes_out) {
  clear_error();
  if (!g || !bytes_out || !valid_kind(kind) || !valid_prec(prec)) {
    set_error("lq_field_bytes: invalid argument");
    return LQ_ERR_ARG;
  }
  *bytes_out = field_bytes(*g, kind, prec);
  return LQ_OK;
}

lq_status lq_field_alloc(const lq_geom* g, int kind, int prec, void* stream, lq_field** out) {
  clear_error();
  if (!g || !out || !valid_kind(kind) || !valid_prec(prec)) {
    set_error("lq_field_alloc: invalid argument (kind %d, prec %d)", kind, prec);
    return LQ_ERR_ARG;
  }
  lq_field* f = new (std::nothrow) lq_field;
  if (!f) {
    set_error("lq_field_alloc: host allocation failed");
    return LQ_ERR_OOM;
  }
  f->geom = *g;
  f->kind = kind;
  f->prec = prec;
  f->bytes = field_bytes(*g, kind, prec);
  f->owned = true;
  lq_status st = scratch_alloc(&f->ptr, f->bytes, as_stream(stream), "lq_field_alloc");
  if (st != LQ_OK) {
    delete f;
    return st;
  }
  *out = f;
  return LQ_OK;
}

lq_status lq_field_wrap(const lq_geom* g, int kind, int prec, void* dev_ptr, size_t bytes, lq_field** out) {
  clear_error();
  if (!g || !out || !dev_ptr || !valid_kind(kind) || !valid_prec(prec)) {
    set_error("lq_field_wrap: invalid argument");
    return LQ_ERR_ARG;
  }
  if (((uintptr_t)dev_ptr) & 15u) {
    set_error("lq_field_wrap: device pointer must be 16-byte aligned");
    return LQ_ERR_ARG;
  }
  size_t need = field_bytes(*g, kind, prec);
  if (bytes < need) {
    set_error("lq_field_wrap: %zu bytes given, %zu needed", bytes, need);
    return LQ_ERR_ARG;
  }
  lq_field* f = new (std::nothrow) lq_field;
  if (!f) {
    set_error("lq_field_wrap: host allocation failed");
    return LQ_ERR_OOM;
  }
  f->geom = *g;
  f->kind = kind;
  f->prec = prec;
  f->ptr = dev_ptr;
  f->bytes = need;
  f->owned = false;
  *out = f;
  return LQ_OK;
}

lq_status lq_field_free(lq_field* f) {
  clear_error();
  if (!f) return LQ_OK;
  lq_status st = LQ_OK;
  if (f->owned && f->ptr) st = cuda_check(cudaFree(f->ptr), "lq_field_free");
  delete f;
  return st;
}

lq_status lq_field_device_ptr(const lq_field* f, void** ptr_out) {
  clear_error();
  if (!f || !ptr_out) {
    set_error("lq_field_device_ptr: NULL argument");
    return LQ_ERR_ARG;
  }
  *ptr_out = f->ptr;
  return LQ_OK;
}

lq_status lq_field_upload(lq_field* f, const void* host_aos, void* stream) {
  clear_error();
  if (!f || !host_aos) {
    set_error("lq_field_upload: NULL argument");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  void* stage = nullptr;
  lq_status st = scratch_alloc(&stage, f->bytes, s, "lq_field_upload");
  if (st != LQ_OK) return st;
  st = cuda_check(cudaMemcpyAsync(stage, host_aos, f->bytes, cudaMemcpyHostToDevice, s), "lq_field_upload copy");
  if (st == LQ_OK) st = transpose(stage, f->ptr, f, true, s);
  scratch_free(stage, s);
  lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_field_upload sync");
  return st != LQ_OK ? st : st2;
}

lq_status lq_field_download(const lq_field* f, void* host_aos, void* stream) {
  clear_error();
  if (!f || !host_aos) {
    set_error("lq_field_download: NULL argument");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  void* stage = nullptr;
  lq_status st = scratch_alloc(&stage, f->bytes, s, "lq_field_download");
  if (st != LQ_OK) return st;
  st = transpose(f->ptr, stage, f, false, s);
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpyAsync(host_aos, stage, f->bytes, cudaMemcpyDeviceToHost, s), "lq_field_download copy");
  scratch_free(stage, s);
  lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_field_download sync");
  return st != LQ_OK ? st : st2;
}

lq_status lq_free_all(void) {
  clear_error();
  std::vector<void (*)()> fns;
  {
    std::lock_guard<std::mutex> lk(g_release_mu);
    fns = release_list();
  }
  for (auto fn : fns) fn();
  return LQ_OK;
}

}  // extern "C"
