// Geometry, field handles, host<->device transfers, error reporting and the
// device-storage release of liblqcd (device residency API of Winter,
// "Accelerating QDP++ using GPUs", Sec. 5; coalesced layout, Sec. 8).
#include <cstdarg>
#include <cstdlib>
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

// Host-side fault injection for tests of the error paths: with the
// environment variable LQ_FAULT_INJECT=alloc every library scratch allocation
// fails with LQ_ERR_OOM before any CUDA call is made.
static bool inject_alloc_failure() {
  const char* v = getenv("LQ_FAULT_INJECT");
  return v && strcmp(v, "alloc") == 0;
}

// The library's own stream-ordered memory pool per device.  Unlike the
// device's default pool (release threshold 0: memory goes back to the driver
// at every synchronisation) it keeps freed memory for the next call, so
// repeated smearing / transfer calls do not re-map gigabytes each time;
// lq_free_all trims it.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {nullptr};

static lq_status library_pool(cudaMemPool_t* out) {
  const int dev = current_device();
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return LQ_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    lq_status st = cuda_check(cudaMemPoolCreate(&pool, &props), "memory pool");
    if (st != LQ_OK) return st;
    unsigned long long keep = ~0ull;
    st = cuda_check(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "memory pool threshold");
    if (st != LQ_OK) {
      cudaMemPoolDestroy(pool);
      return st;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return LQ_OK;
}

static void trim_pools() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < 64; ++d)
    if (g_pool[d]) cudaMemPoolTrimTo(g_pool[d], 0);
}

lq_status scratch_alloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  if (inject_alloc_failure()) {
    set_error("%s: allocation of %zu bytes failed (fault injected by LQ_FAULT_INJECT=alloc)", what, bytes);
    return LQ_ERR_OOM;
  }
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = nullptr;
  lq_status pst = library_pool(&pool);
  if (pst != LQ_OK) return pst;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
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
// A CTA moves a tile of kTileSites consecutive sites: the AoS side of the tile
// is one contiguous run of kTileSites * per_site elements, each SoA plane gets
// a contiguous run of kTileSites elements; the tile goes through shared memory
// so that both global sides are accessed with consecutive addresses (the tile
// rows are padded to per_site + 1 elements against shared-memory bank conflicts).
constexpr int kTileSites = 64;
constexpr int kTileThreads = 256;

template <typename E>
__global__ void __launch_bounds__(kTileThreads) aos_to_soa(const E* __restrict__ aos, E* __restrict__ soa, long long V,
                                                           int per_site, long long s_begin, long long s_end) {
  extern __shared__ __align__(16) unsigned char tile_raw[];
  E* tile = reinterpret_cast<E*>(tile_raw);  // [kTileSites][per_site + 1]
  const int ld = per_site + 1;
  const long long s0 = s_begin + (long long)blockIdx.x * kTileSites;
  const int ns = (int)min((long long)kTileSites, s_end - s0);
  const int n = ns * per_site;
  const E* src = aos + s0 * per_site;
  for (int i = threadIdx.x; i < n; i += kTileThreads) {
    const int j = i / per_site, c = i - j * per_site;
    tile[j * ld + c] = src[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kTileThreads) {
    const int c = i / ns, j = i - c * ns;
    soa[(long long)c * V + s0 + j] = tile[j * ld + c];
  }
}
template <typename E>
__global__ void __launch_bounds__(kTileThreads) soa_to_aos(const E* __restrict__ soa, E* __restrict__ aos, long long V,
                                                           int per_site, long long s_begin, long long s_end) {
  extern __shared__ __align__(16) unsigned char tile_raw[];
  E* tile = reinterpret_cast<E*>(tile_raw);
  const int ld = per_site + 1;
  const long long s0 = s_begin + (long long)blockIdx.x * kTileSites;
  const int ns = (int)min((long long)kTileSites, s_end - s0);
  const int n = ns * per_site;
  for (int i = threadIdx.x; i < n; i += kTileThreads) {
    const int c = i / ns, j = i - c * ns;
    tile[j * ld + c] = soa[(long long)c * V + s0 + j];
  }
  __syncthreads();
  E* dst = aos + s0 * per_site;
  for (int i = threadIdx.x; i < n; i += kTileThreads) {
    const int j = i / per_site, c = i - j * per_site;
    dst[i] = tile[j * ld + c];
  }
}

lq_status transpose_range(const void* src, void* dst, const lq_geom& g, int kind, int prec, bool to_soa,
                          long long s_begin, long long s_end, cudaStream_t s) {
  const long long V = g.volume;
  const int per_site = ndir_of(kind) * ncomp_of(kind);
  const size_t eb = elem_bytes(kind, prec);
  const unsigned blocks = (unsigned)((s_end - s_begin + kTileSites - 1) / kTileSites);
  if (blocks == 0) return LQ_OK;
  const size_t smem = (size_t)kTileSites * (per_site + 1) * eb;  // <= 64 * 37 * 16 B = 37.9 KB
#define LQ_T(E)                                                                                            \
  if (to_soa)                                                                                              \
    aos_to_soa<E><<<blocks, kTileThreads, smem, s>>>((const E*)src, (E*)dst, V, per_site, s_begin, s_end);  \
  else                                                                                                     \
    soa_to_aos<E><<<blocks, kTileThreads, smem, s>>>((const E*)src, (E*)dst, V, per_site, s_begin, s_end);
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

static lq_status transpose(const void* src, void* dst, const lq_field* f, bool to_soa, cudaStream_t s) {
  return transpose_range(src, dst, f->geom, f->kind, f->prec, to_soa, 0, f->geom.volume, s);
}

void* host_device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
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
  if (const void* dv = host_device_view(host_aos)) {   // page-locked: the transpose reads it directly
    lq_status st = transpose(dv, f->ptr, f, true, s);
    lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_field_upload sync");
    return st != LQ_OK ? st : st2;
  }
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
  if (void* dv = host_device_view(host_aos)) {   // page-locked: the transpose writes it directly
    lq_status st = transpose(f->ptr, dv, f, false, s);
    lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_field_download sync");
    return st != LQ_OK ? st : st2;
  }
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

namespace {
struct FieldFileHeader {
  char magic[8];
  int version;
  int kind;
  int prec;
  int dims[4];
  int reserved;
  long long bytes;
};
static_assert(sizeof(FieldFileHeader) == 48, "checkpoint header is 48 bytes");
}  // namespace

lq_status lq_field_save(const lq_field* f, const char* path, void* stream) {
  clear_error();
  if (!f || !path) {
    set_error("lq_field_save: NULL argument");
    return LQ_ERR_ARG;
  }
  std::vector<char> host;
  try {
    host.resize(f->bytes);
  } catch (...) {
    set_error("lq_field_save: host allocation of %zu bytes failed", f->bytes);
    return LQ_ERR_OOM;
  }
  lq_status st = lq_field_download(f, host.data(), stream);
  if (st != LQ_OK) return st;
  FieldFileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "LQFIELD1", 8);
  h.version = 1;
  for (int i = 0; i < 4; ++i) h.dims[i] = f->geom.dims[i];
  h.kind = f->kind;
  h.prec = f->prec;
  h.bytes = (long long)f->bytes;
  FILE* fp = fopen(path, "wb");
  if (!fp) {
    set_error("lq_field_save: cannot open %s for writing", path);
    return LQ_ERR_ARG;
  }
  const bool ok = fwrite(&h, sizeof(h), 1, fp) == 1 && fwrite(host.data(), 1, host.size(), fp) == host.size();
  const bool closed = fclose(fp) == 0;
  if (!ok || !closed) {
    set_error("lq_field_save: writing %s failed", path);
    return LQ_ERR_ARG;
  }
  return LQ_OK;
}

lq_status lq_field_load(lq_field* f, const char* path, void* stream) {
  clear_error();
  if (!f || !path) {
    set_error("lq_field_load: NULL argument");
    return LQ_ERR_ARG;
  }
  FILE* fp = fopen(path, "rb");
  if (!fp) {
    set_error("lq_field_load: cannot open %s", path);
    return LQ_ERR_ARG;
  }
  FieldFileHeader h;
  if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "LQFIELD1", 8) != 0 || h.version != 1) {
    fclose(fp);
    set_error("lq_field_load: %s is not a liblqcd field checkpoint", path);
    return LQ_ERR_ARG;
  }
  bool same = h.kind == f->kind && h.prec == f->prec && h.bytes == (long long)f->bytes;
  for (int i = 0; i < 4; ++i) same = same && h.dims[i] == f->geom.dims[i];
  if (!same) {
    fclose(fp);
    set_error("lq_field_load: %s holds dims %dx%dx%dx%d kind %d prec %d, the field differs", path, h.dims[0],
              h.dims[1], h.dims[2], h.dims[3], h.kind, h.prec);
    return LQ_ERR_GEOM;
  }
  std::vector<char> host;
  try {
    host.resize(f->bytes);
  } catch (...) {
    fclose(fp);
    set_error("lq_field_load: host allocation of %zu bytes failed", f->bytes);
    return LQ_ERR_OOM;
  }
  const bool ok = fread(host.data(), 1, host.size(), fp) == host.size();
  fclose(fp);
  if (!ok) {
    set_error("lq_field_load: %s is truncated", path);
    return LQ_ERR_ARG;
  }
  return lq_field_upload(f, host.data(), stream);
}

lq_status lq_free_all(void) {
  clear_error();
  std::vector<void (*)()> fns;
  {
    std::lock_guard<std::mutex> lk(g_release_mu);
    fns = release_list();
  }
  for (auto fn : fns) fn();
  cudaDeviceSynchronize();
  trim_pools();
  return LQ_OK;
}

}  // extern "C"
