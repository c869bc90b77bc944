// Batched stout smearing of many independent lattices of uneven sizes: one
// persistent launch per step walks a device work list of (config, direction,
// tile) items handed out by an atomic counter; the n-step sequence can be a
// replayed CUDA graph.  Block size and sites per thread (the tile) come from
// the auto-tuner (thread geometry of Winter, "Accelerating QDP++ using GPUs",
// Sec. 4.4).  Per-link arithmetic is stout_link(), so every configuration's
// result is bit-identical to a separate lq_stout_smear call.
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "lq_internal.h"
#include "stout_core.cuh"

namespace lq {

struct BatchDesc {
  GeomArgs g;
  void* a;               // the caller's links
  long long b_off;       // byte offset of this config's slice of the workspace
  long long item_begin;  // first work item of this config
  int tiles_per_dir;
  int pad;
};

struct MuList4 {
  int mu[4];
};

template <typename R, bool REPRO>
__device__ __forceinline__ void stout_batch_body(const BatchDesc* __restrict__ D, int n_cfg, long long n_items,
                                                 char* work, unsigned long long* __restrict__ counter, int parity, R rho,
                                                 unsigned dirs, int nsite, int nd, const MuList4& ml,
                                                 long long& item_s) {
  typedef typename vec2<R>::type V2;
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= n_items) return;
    int lo = 0, hi = n_cfg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (D[mid].item_begin <= item) lo = mid;
      else hi = mid - 1;
    }
    const GeomArgs g = D[lo].g;
    const long long local = item - D[lo].item_begin;
    // the smeared directions of one tile are consecutive items, so the
    // direction sweeps of a tile share cached lines
    const int mi = (int)(local % nd);
    const long long tile = local / nd;
    const int mu = mi == 0 ? ml.mu[0] : (mi == 1 ? ml.mu[1] : (mi == 2 ? ml.mu[2] : ml.mu[3]));
    V2* const b = (V2*)(work + D[lo].b_off);
    const V2* in = parity ? (const V2*)b : (const V2*)D[lo].a;
    V2* out = parity ? (V2*)D[lo].a : b;
    const long long V = g.V;
    for (int k = 0; k < nsite; ++k) {
      const long long sl = (tile * nsite + k) * blockDim.x + threadIdx.x;
      if (sl >= V) break;
      const int s = (int)sl;
      int c[4];
      site_coords(g, s, c);
      const M3<R> Up = stout_link<R>(in, g, s, c, mu, dirs, rho, REPRO);
      st_m3<R>(out + (long long)mu * 9 * V + s, V, Up);
    }
  }
}

// FP32 links: capped at 80 registers (24 resident warps per SM instead of 16;
// ptxas reports 24 bytes of spill stores per thread).
template <bool REPRO>
__global__ void __maxnreg__(80) k_stout_batch_f32(const BatchDesc* __restrict__ D, int n_cfg, long long n_items,
                                                  char* work, unsigned long long* __restrict__ counter, int parity,
                                                  float rho, unsigned dirs, int nsite, int nd, MuList4 ml) {
  __shared__ long long item_s;
  stout_batch_body<float, REPRO>(D, n_cfg, n_items, work, counter, parity, rho, dirs, nsite, nd, ml, item_s);
}

template <bool REPRO>
__global__ void __launch_bounds__(256) k_stout_batch_f64(const BatchDesc* __restrict__ D, int n_cfg,
                                                         long long n_items, char* work,
                                                         unsigned long long* __restrict__ counter, int parity,
                                                         double rho, unsigned dirs, int nsite, int nd, MuList4 ml) {
  __shared__ long long item_s;
  stout_batch_body<double, REPRO>(D, n_cfg, n_items, work, counter, parity, rho, dirs, nsite, nd, ml, item_s);
}

// Descriptor table of one (fields, dims, tile, dirs) combination: where each
// configuration's work items start and where its half of the double buffer
// lies in a workspace of work_bytes.  It holds no workspace itself.
struct BatchLayout {
  std::vector<BatchDesc> host;
  BatchDesc* dev = nullptr;
  long long n_items = 0;
  size_t work_bytes = 0;
};

// A recorded n-step graph owns its descriptors, workspace and counters.
struct BatchGraph {
  BatchLayout lay;
  void* work = nullptr;
  unsigned long long* counters = nullptr;  // one per step
  cudaGraphExec_t exec = nullptr;
};

struct LayoutKey {
  std::vector<void*> ptrs;
  std::vector<int> dims;
  int prec, block, nsite, device;
  unsigned dirs;
  bool operator<(const LayoutKey& o) const {
    if (ptrs != o.ptrs) return ptrs < o.ptrs;
    if (dims != o.dims) return dims < o.dims;
    const int a[4] = {prec, block, nsite, device};
    const int b[4] = {o.prec, o.block, o.nsite, o.device};
    for (int i = 0; i < 4; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return dirs < o.dirs;
  }
};

struct GraphKeyB {
  LayoutKey lk;
  int n, reproject;
  double rho;
  bool operator<(const GraphKeyB& o) const {
    if (lk < o.lk) return true;
    if (o.lk < lk) return false;
    if (n != o.n) return n < o.n;
    if (reproject != o.reproject) return reproject < o.reproject;
    return rho < o.rho;
  }
};

// Both caches are bounded; the least recently used entry is evicted.
constexpr size_t kMaxLayouts = 16;
constexpr size_t kMaxBatchGraphs = 4;

template <typename T> struct Lru {
  T v;
  unsigned long long used = 0;
};

static std::mutex g_batch_mu;
static unsigned long long g_batch_tick = 0;
static std::map<LayoutKey, Lru<BatchLayout>>& layout_cache() {
  static std::map<LayoutKey, Lru<BatchLayout>> m;
  return m;
}
static std::map<GraphKeyB, Lru<BatchGraph>>& batch_graph_cache() {
  static std::map<GraphKeyB, Lru<BatchGraph>> m;
  return m;
}
static void free_layout(BatchLayout& l) {
  if (l.dev) cudaFree(l.dev);
  l = BatchLayout();
}
static void free_graph(BatchGraph& p) {
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.counters) cudaFree(p.counters);
  if (p.work) cudaFree(p.work);
  free_layout(p.lay);
  p = BatchGraph();
}
template <typename M, typename F> static void evict_lru(M& m, size_t cap, F free_fn) {
  while (m.size() >= cap) {
    auto old = m.begin();
    for (auto it = m.begin(); it != m.end(); ++it)
      if (it->second.used < old->second.used) old = it;
    free_fn(old->second.v);
    m.erase(old);
  }
}
static void release_batch() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto& kv : layout_cache()) free_layout(kv.second.v);
  layout_cache().clear();
  for (auto& kv : batch_graph_cache()) free_graph(kv.second.v);
  batch_graph_cache().clear();
}

static lq_status make_layout(lq_field* const* links, int n_cfg, unsigned dirs, const TuneChoice& tc,
                             BatchLayout* out) {
  BatchLayout l;
  int nd = 0;
  for (int mu = 0; mu < 4; ++mu) nd += (dirs >> mu) & 1u;
  size_t off = 0;
  long long items = 0;
  const long long tile = (long long)tc.block * tc.nsite;
  for (int i = 0; i < n_cfg; ++i) {
    BatchDesc d;
    std::memset(&d, 0, sizeof(d));
    d.g = geom_args(links[i]->geom);
    d.a = links[i]->ptr;
    d.b_off = (long long)off;
    d.item_begin = items;
    d.tiles_per_dir = (int)((d.g.V + tile - 1) / tile);
    items += (long long)d.tiles_per_dir * nd;
    off += (links[i]->bytes + 255) / 256 * 256;
    l.host.push_back(d);
  }
  l.n_items = items;
  l.work_bytes = off;
  lq_status st = cuda_check(cudaMalloc(&l.dev, sizeof(BatchDesc) * n_cfg), "batch descriptors");
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpy(l.dev, l.host.data(), sizeof(BatchDesc) * n_cfg, cudaMemcpyHostToDevice),
                    "batch descriptor upload");
  if (st != LQ_OK) {
    free_layout(l);
    return st;
  }
  *out = l;
  return LQ_OK;
}

// Records the whole n-step sequence on stream s (also used under capture).
static lq_status batch_sequence(lq_field* const* links, int n_cfg, const BatchLayout& L, void* work,
                                unsigned long long* counters, int n_steps, double rho, unsigned dirs, int reproject,
                                const TuneChoice& tc, int prec, cudaStream_t s) {
  lq_status st = cuda_check(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * n_steps, s), "batch counters");
  if (st) return st;
  const size_t eb = elem_bytes(LQ_LINKS, prec);
  char* const wb = (char*)work;
  for (int i = 0; i < n_cfg; ++i) {
    const size_t db = (size_t)links[i]->geom.volume * 9 * eb;
    for (int mu = 0; mu < 4; ++mu)
      if (!((dirs >> mu) & 1u))
        if ((st = cuda_check(cudaMemcpyAsync(wb + L.host[i].b_off + mu * db, (const char*)links[i]->ptr + mu * db, db,
                                             cudaMemcpyDeviceToDevice, s),
                             "batch pass-through copy")))
          return st;
  }
  int nd = 0;
  MuList4 ml;
  for (int mu = 0; mu < 4; ++mu)
    if ((dirs >> mu) & 1u) ml.mu[nd++] = mu;
  for (int j = nd; j < 4; ++j) ml.mu[j] = 0;
  const int grid = device_sm_count() * (prec == LQ_F64 ? 4 : 8) * 128 / tc.block;
  for (int k = 0; k < n_steps; ++k) {
    const int parity = k & 1;
    unsigned long long* ctr = counters + k;
    if (prec == LQ_F64) {
      if (reproject)
        k_stout_batch_f64<true><<<grid, tc.block, 0, s>>>(L.dev, n_cfg, L.n_items, wb, ctr, parity, rho, dirs, tc.nsite, nd, ml);
      else
        k_stout_batch_f64<false><<<grid, tc.block, 0, s>>>(L.dev, n_cfg, L.n_items, wb, ctr, parity, rho, dirs, tc.nsite, nd, ml);
    } else {
      if (reproject)
        k_stout_batch_f32<true><<<grid, tc.block, 0, s>>>(L.dev, n_cfg, L.n_items, wb, ctr, parity, (float)rho, dirs, tc.nsite, nd, ml);
      else
        k_stout_batch_f32<false><<<grid, tc.block, 0, s>>>(L.dev, n_cfg, L.n_items, wb, ctr, parity, (float)rho, dirs, tc.nsite, nd, ml);
    }
    if ((st = launch_check("k_stout_batch"))) return st;
  }
  if (n_steps % 2 == 1) {
    for (int i = 0; i < n_cfg; ++i) {
      const size_t db = (size_t)links[i]->geom.volume * 9 * eb;
      for (int mu = 0; mu < 4; ++mu)
        if ((dirs >> mu) & 1u)
          if ((st = cuda_check(cudaMemcpyAsync((char*)links[i]->ptr + mu * db, wb + L.host[i].b_off + mu * db, db,
                                               cudaMemcpyDeviceToDevice, s),
                               "batch result copy")))
            return st;
    }
  }
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_stout_smear_batch(lq_field* const* links, int n_cfg, double rho, int n_steps, unsigned dirs_mask,
                                          const lq_stout_opts* opts, void* stream) {
  clear_error();
  if (!links || n_cfg < 1) {
    set_error("lq_stout_smear_batch: need n_cfg >= 1 fields");
    return LQ_ERR_ARG;
  }
  lq_status st;
  if ((st = check_dirs(dirs_mask, "lq_stout_smear_batch"))) return st;
  if (!(rho >= 0.0) || rho > 1e6 || n_steps < 0) {
    set_error("lq_stout_smear_batch: rho must be finite >= 0 and n_steps >= 0");
    return LQ_ERR_ARG;
  }
  for (int i = 0; i < n_cfg; ++i) {
    if ((st = check_links(links[i], "lq_stout_smear_batch"))) return st;
    if (links[i]->prec != links[0]->prec) {
      set_error("lq_stout_smear_batch: all fields must share one precision");
      return LQ_ERR_GEOM;
    }
    for (int j = 0; j < i; ++j)
      if (links[j]->ptr == links[i]->ptr) {
        set_error("lq_stout_smear_batch: fields %d and %d alias", j, i);
        return LQ_ERR_ARG;
      }
  }
  const lq_stout_opts* o = (opts && opts->struct_size >= (int)sizeof(lq_stout_opts)) ? opts : nullptr;
  if (n_steps == 0) return LQ_OK;
  const int prec = links[0]->prec;
  const int reproject = (o && o->reproject >= 0) ? o->reproject : (prec == LQ_F32 ? 1 : 0);
  cudaStream_t s = as_stream(stream);
  TuneChoice tc = stout_default_choice(prec);
  if (o && o->block > 0) {
    if (o->block % 32 != 0 || o->block > 256) {
      set_error("lq_stout_smear_batch: block must be a multiple of 32 in [32, 256]");
      return LQ_ERR_ARG;
    }
    tc.block = o->block;
    tc.nsite = o->sites_per_thread > 0 ? o->sites_per_thread : 1;
  } else if (tune_enabled()) {
    // the tile shape tuned for the largest member is used for the whole batch
    int big = 0;
    for (int i = 1; i < n_cfg; ++i)
      if (links[i]->geom.volume > links[big]->geom.volume) big = i;
    if ((st = stout_choose(links[big], rho, dirs_mask, reproject, nullptr, s, &tc))) return st;
    if (tc.variant != 1) tc = stout_default_choice(prec);  // the batch kernel reads through L1/L2
  }
  const bool use_graph = o && o->use_graph;
  register_cache_release(release_batch);

  LayoutKey lkey;
  for (int i = 0; i < n_cfg; ++i) {
    lkey.ptrs.push_back(links[i]->ptr);
    for (int d = 0; d < 4; ++d) lkey.dims.push_back(links[i]->geom.dims[d]);
  }
  lkey.prec = prec;
  lkey.block = tc.block;
  lkey.nsite = tc.nsite;
  lkey.device = current_device();
  lkey.dirs = dirs_mask;

  std::lock_guard<std::mutex> lk(g_batch_mu);
  const unsigned long long now = ++g_batch_tick;
  if (use_graph) {
    GraphKeyB gkey{lkey, n_steps, reproject, rho};
    auto it = batch_graph_cache().find(gkey);
    if (it == batch_graph_cache().end()) {
      evict_lru(batch_graph_cache(), kMaxBatchGraphs, free_graph);
      BatchGraph p;
      if ((st = make_layout(links, n_cfg, dirs_mask, tc, &p.lay))) return st;
      if ((st = cuda_check(cudaMalloc(&p.work, p.lay.work_bytes), "batch graph workspace")) ||
          (st = cuda_check(cudaMalloc(&p.counters, sizeof(unsigned long long) * n_steps), "batch counters"))) {
        free_graph(p);
        return st;
      }
      cudaStream_t cap;
      if ((st = cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "batch graph stream"))) {
        free_graph(p);
        return st;
      }
      cudaGraph_t graph = nullptr;
      st = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "batch graph capture");
      if (!st) {
        lq_status st_run = batch_sequence(links, n_cfg, p.lay, p.work, p.counters, n_steps, rho, dirs_mask,
                                          reproject, tc, prec, cap);
        lq_status st_end = cuda_check(cudaStreamEndCapture(cap, &graph), "batch graph end capture");
        st = st_run ? st_run : st_end;
      }
      if (!st) st = cuda_check(cudaGraphInstantiate(&p.exec, graph, 0), "batch graph instantiate");
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      if (st) {
        free_graph(p);
        return st;
      }
      it = batch_graph_cache().emplace(gkey, Lru<BatchGraph>{p, now}).first;
    }
    it->second.used = now;
    return cuda_check(cudaGraphLaunch(it->second.v.exec, s), "batch graph launch");
  }
  auto it = layout_cache().find(lkey);
  if (it == layout_cache().end()) {
    evict_lru(layout_cache(), kMaxLayouts, free_layout);
    BatchLayout l;
    if ((st = make_layout(links, n_cfg, dirs_mask, tc, &l))) return st;
    it = layout_cache().emplace(lkey, Lru<BatchLayout>{l, now}).first;
  }
  it->second.used = now;
  // workspace and counters stream-ordered from the library pool, per call
  void* work = nullptr;
  void* counters = nullptr;
  if ((st = scratch_alloc(&work, it->second.v.work_bytes, s, "lq_stout_smear_batch workspace"))) return st;
  if ((st = scratch_alloc(&counters, sizeof(unsigned long long) * n_steps, s, "lq_stout_smear_batch counters"))) {
    scratch_free(work, s);
    return st;
  }
  st = batch_sequence(links, n_cfg, it->second.v, work, (unsigned long long*)counters, n_steps, rho, dirs_mask,
                      reproject, tc, prec, s);
  scratch_free(counters, s);
  scratch_free(work, s);
  return st;
}
