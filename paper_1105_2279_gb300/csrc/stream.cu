// Stout smearing of links held in host memory, with the host<->device
// transfers pipelined against the smearing.  The lattice is cut into slabs of
// whole t-slices (contiguous site ranges in the lexicographic order, so a slab
// is one contiguous piece of the host AoS array and of every SoA plane).
//   upload streams:  per slab, H2D copy into an AoS staging buffer, then (on
//                    a second stream) the AoS -> SoA transpose of that slab;
//                    event up[i].
//   compute stream:  step 1 of slab i waits for up[i-1], up[i], up[i+1] (the
//                    staples reach one t-slice into each neighbour); after
//                    the last step of slab i, event fin[i].
//   download streams: per slab, waits for fin[i], transposes the slab back
//                    into the staging buffer and (on a second stream) copies
//                    it to the host.
// Step k of a slab reads field (k-1)%2 and writes field k%2, so (k, i) must
// follow (k-1, j) for the slabs j next to i (their reads of field k%2 and
// the values it reads).  The first two and the last two steps run as
// (step, slab) items in the order of the key 2k + d(i), d(i) the cyclic
// distance of slab i from slab 0: neighbouring slabs differ by at most 1 in
// d, so every item comes after those it depends on, and the wavefront lets
// the slabs near slab 0 finish about d_max / 2 steps before the farthest
// ones, which spreads the downloads over the last steps.  The steps in
// between are whole-lattice launches.  Uploads go in the order of d as well.
// (Winter, "Accelerating QDP++ using GPUs", Sec. 4.3 moves whole fields
// between host and device on demand; here the device layout stays fixed and
// the transfers run behind the arithmetic.)
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lq_internal.h"

using namespace lq;

namespace {

// Copies and transposes of a direction run on separate streams, so that the
// transpose of one slab overlaps the host-link copy of the next (uploads) or
// of the previous one (downloads): a slab's copy takes ~1 ms over the host
// link, its transpose ~0.1 ms on the SMs.
struct Streams {
  cudaStream_t up = nullptr, down = nullptr, upx = nullptr, downx = nullptr;
  std::vector<cudaEvent_t> ev;
  ~Streams() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t q : {up, down, upx, downx})
      if (q) cudaStreamDestroy(q);
  }
  // The transfer streams get the highest priority: their transposes are short
  // and must not queue behind the tens of thousands of pending blocks of a
  // step kernel (the block scheduler serves higher-priority streams first).
  lq_status make(int n_events) {
    int least = 0, greatest = 0;
    lq_status st = cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    if (st == LQ_OK)
      st = cuda_check(cudaStreamCreateWithPriority(&up, cudaStreamNonBlocking, greatest), "upload stream");
    if (st == LQ_OK)
      st = cuda_check(cudaStreamCreateWithPriority(&down, cudaStreamNonBlocking, greatest), "download stream");
    if (st == LQ_OK)
      st = cuda_check(cudaStreamCreateWithPriority(&upx, cudaStreamNonBlocking, greatest), "upload transpose stream");
    if (st == LQ_OK)
      st = cuda_check(cudaStreamCreateWithPriority(&downx, cudaStreamNonBlocking, greatest),
                      "download transpose stream");
    for (int i = 0; i < n_events && st == LQ_OK; ++i) {
      cudaEvent_t e;
      st = cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "pipeline event");
      if (st == LQ_OK) ev.push_back(e);
    }
    return st;
  }
};

int slab_count(int Lt, int n_chunks) {
  int nc = n_chunks > 0 ? n_chunks : 16;
  return nc > Lt ? Lt : nc;
}

int cyclic_distance(int i, int nc) { return std::min(i, nc - i); }

// Optional timeline: with LQ_PIPELINE_TRACE=<file>, timing events are recorded
// around every copy, transpose and step launch, and one line per operation
// ("what slab step start_ms end_ms", relative to the call's start on the
// compute stream) is appended to <file> after the call has synchronised.
struct Trace {
  const char* path = nullptr;
  cudaEvent_t t0 = nullptr;
  struct Op {
    char what[12];
    int slab, step;
    cudaEvent_t a, b;
    bool owns;
  };
  std::vector<Op> ops;
  Trace() {
    path = getenv("LQ_PIPELINE_TRACE");
    if (path && !*path) path = nullptr;
  }
  void begin(cudaStream_t s) {
    if (!path) return;
    cudaEventCreate(&t0);
    cudaEventRecord(t0, s);
  }
  int open(const char* what, int slab, int step, cudaStream_t s) {
    if (!path) return -1;
    Op o;
    snprintf(o.what, sizeof(o.what), "%s", what);
    o.slab = slab;
    o.step = step;
    cudaEventCreate(&o.a);
    cudaEventCreate(&o.b);
    o.owns = true;
    cudaEventRecord(o.a, s);
    ops.push_back(o);
    return (int)ops.size() - 1;
  }
  // another operation that ran inside the same launch as op `id`
  void alias(const char* what, int slab, int step, int id) {
    if (id < 0) return;
    Op o = ops[id];
    snprintf(o.what, sizeof(o.what), "%s", what);
    o.slab = slab;
    o.step = step;
    o.owns = false;
    ops.push_back(o);
  }
  void close(int id, cudaStream_t s) {
    if (id >= 0) cudaEventRecord(ops[id].b, s);
  }
  void write() {
    if (!path) return;
    FILE* fp = fopen(path, "a");
    for (const Op& o : ops) {
      float a = 0, b = 0;
      if (fp && cudaEventElapsedTime(&a, t0, o.a) == cudaSuccess && cudaEventElapsedTime(&b, t0, o.b) == cudaSuccess)
        fprintf(fp, "%s %d %d %.4f %.4f\n", o.what, o.slab, o.step, a, b);
    }
    if (fp) {
      fprintf(fp, "end -1 -1 0 0\n");
      fclose(fp);
    }
  }
  ~Trace() {
    for (Op& o : ops)
      if (o.owns) {
        cudaEventDestroy(o.a);
        cudaEventDestroy(o.b);
      }
    if (t0) cudaEventDestroy(t0);
  }
};

}  // namespace

extern "C" lq_status lq_stout_smear_host(const void* host_in, void* host_out, const lq_geom* geom, int prec,
                                         double rho, int n_steps, unsigned dirs_mask, int n_chunks,
                                         double* plaq_out, const lq_stout_opts* opts, void* stream) {
  clear_error();
  if (!host_in || !host_out || !geom) {
    set_error("lq_stout_smear_host: NULL argument");
    return LQ_ERR_ARG;
  }
  if (!valid_prec(prec)) {
    set_error("lq_stout_smear_host: precision %d is not LQ_F32 or LQ_F64", prec);
    return LQ_ERR_ARG;
  }
  lq_status st = check_dirs(dirs_mask, "lq_stout_smear_host");
  if (st != LQ_OK) return st;
  if (!(rho >= 0.0) || rho > 1e6 || n_steps < 0 || n_chunks < 0) {
    set_error("lq_stout_smear_host: need finite rho >= 0, n_steps >= 0, n_chunks >= 0");
    return LQ_ERR_ARG;
  }
  const lq_stout_opts* o = (opts && opts->struct_size >= (int)sizeof(lq_stout_opts)) ? opts : nullptr;
  if (opts && !o && opts->struct_size != 0) {
    set_error("lq_stout_smear_host: opts->struct_size %d < sizeof(lq_stout_opts)", opts->struct_size);
    return LQ_ERR_ARG;
  }
  const lq_geom& g = *geom;
  const size_t bytes = field_bytes(g, LQ_LINKS, prec);
  const size_t eb = elem_bytes(LQ_LINKS, prec);
  const long long V = g.volume;
  const long long slice = V / g.dims[3];
  const int nc = slab_count(g.dims[3], n_chunks);
  std::vector<long long> sb(nc + 1);
  for (int i = 0; i <= nc; ++i) sb[i] = slice * (long long)((long long)g.dims[3] * i / nc);
  cudaStream_t s = as_stream(stream);
  const int reproject = (o && o->reproject >= 0) ? o->reproject : (prec == LQ_F32 ? 1 : 0);
  // launch shape: explicit, else a cached tuning result, else the default
  TuneChoice tc = stout_default_choice(prec);
  if (o && o->block > 0) {
    tc.block = o->block;
    tc.nsite = o->sites_per_thread > 0 ? o->sites_per_thread : 1;
  } else if (tune_enabled()) {
    TuneChoice c;
    if (tune_get("stout", prec, g.dims, dirs_mask, &c) && c.variant != 2) tc = c;
  }
  if (tc.block % 32 != 0 || tc.block < 32 || tc.block > 256) {
    set_error("lq_stout_smear_host: block %d must be a multiple of 32 in [32, 256]", tc.block);
    return LQ_ERR_ARG;
  }

  Streams ps;
  if ((st = ps.make(4 * nc + 3)) != LQ_OK) return st;
  cudaEvent_t* up = ps.ev.data();            // slab i transposed in (and its pass-through copies)
  cudaEvent_t* fin = ps.ev.data() + nc;      // slab i's last step done
  cudaEvent_t* copied = ps.ev.data() + 2 * nc;   // slab i copied in
  cudaEvent_t* out_ready = ps.ev.data() + 3 * nc;  // slab i transposed out
  cudaEvent_t start = ps.ev[4 * nc], done = ps.ev[4 * nc + 1], plaq_ready = ps.ev[4 * nc + 2];

  void* f[2] = {nullptr, nullptr};
  void* stage = nullptr;
  if (st == LQ_OK) st = scratch_alloc(&f[0], bytes, s, "lq_stout_smear_host field");
  if (st == LQ_OK && n_steps > 0) st = scratch_alloc(&f[1], bytes, s, "lq_stout_smear_host work field");
  if (st == LQ_OK) st = scratch_alloc(&stage, bytes, s, "lq_stout_smear_host staging");
  Trace tr;
  tr.begin(s);
  // the side streams start after the allocations (and all earlier work) on s
  if (st == LQ_OK) st = cuda_check(cudaEventRecord(start, s), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.up, start, 0), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.down, start, 0), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.upx, start, 0), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.downx, start, 0), "pipeline start");

  const size_t site_bytes = 4 * 9 * eb;
  const size_t plane = (size_t)V * eb;
  std::vector<int> by_distance(nc);
  for (int i = 0; i < nc; ++i) by_distance[i] = i;
  std::stable_sort(by_distance.begin(), by_distance.end(),
                   [nc](int a, int b) { return cyclic_distance(a, nc) < cyclic_distance(b, nc); });
  for (int i : by_distance) {
    if (st != LQ_OK) break;
    const size_t off = (size_t)sb[i] * site_bytes, len = (size_t)(sb[i + 1] - sb[i]) * site_bytes;
    int t = tr.open("h2d", i, 0, ps.up);
    st = cuda_check(cudaMemcpyAsync((char*)stage + off, (const char*)host_in + off, len, cudaMemcpyHostToDevice,
                                    ps.up),
                    "lq_stout_smear_host upload");
    tr.close(t, ps.up);
    if (st == LQ_OK) st = cuda_check(cudaEventRecord(copied[i], ps.up), "pipeline copy event");
    if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.upx, copied[i], 0), "pipeline wait");
    t = tr.open("to_soa", i, 0, ps.upx);
    if (st == LQ_OK) st = transpose_range(stage, f[0], g, LQ_LINKS, prec, true, sb[i], sb[i + 1], ps.upx);
    tr.close(t, ps.upx);
    // links outside dirs are never written: the work field needs them too
    for (int mu = 0; mu < 4 && st == LQ_OK && n_steps > 0; ++mu)
      if (!((dirs_mask >> mu) & 1u))
        for (int c = 0; c < 9 && st == LQ_OK; ++c) {
          const size_t po = (size_t)(mu * 9 + c) * plane + (size_t)sb[i] * eb;
          st = cuda_check(cudaMemcpyAsync((char*)f[1] + po, (const char*)f[0] + po, (size_t)(sb[i + 1] - sb[i]) * eb,
                                          cudaMemcpyDeviceToDevice, ps.upx),
                          "lq_stout_smear_host pass-through copy");
        }
    if (st == LQ_OK) st = cuda_check(cudaEventRecord(up[i], ps.upx), "pipeline upload event");
  }

  // (step, slab) items: the first two and the last two steps in wavefront
  // order (they overlap the uploads and the downloads), the steps between as
  // whole-lattice launches (i = -1), which avoid the per-launch tail and the
  // cold slab boundaries of slab launches
  struct Item {
    int key, k, i;
  };
  std::vector<Item> items;
  auto wave = [&](int k_lo, int k_hi) {
    std::vector<Item> w;
    for (int k = k_lo; k <= k_hi; ++k)
      for (int i = 0; i < nc; ++i) w.push_back({2 * k + cyclic_distance(i, nc), k, i});
    std::stable_sort(w.begin(), w.end(), [](const Item& a, const Item& b) { return a.key < b.key; });
    items.insert(items.end(), w.begin(), w.end());
  };
  if (n_steps <= 4) {
    wave(1, n_steps);
  } else {
    wave(1, 2);
    for (int k = 3; k <= n_steps - 2; ++k) items.push_back({0, k, -1});
    wave(n_steps - 1, n_steps);
  }
  std::vector<int> done_order;   // slabs in the order their final field is complete
  if (n_steps == 0)
    for (int i : by_distance) {
      if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(s, up[i], 0), "pipeline wait");
      if (st == LQ_OK) st = cuda_check(cudaEventRecord(fin[i], s), "pipeline final event");
      done_order.push_back(i);
    }
  // items of one wavefront key are independent: they run as one launch of the
  // multi-segment step kernel (one grid tail per key instead of per slab)
  for (size_t a = 0; a < items.size() && st == LQ_OK;) {
    if (items[a].i < 0) {   // whole-lattice step
      const int k = items[a].k;
      const int t = tr.open("step", -1, k, s);
      st = stout_step_range(f[(k - 1) % 2], f[k % 2], g, prec, rho, dirs_mask, reproject, tc, 0, V, s);
      tr.close(t, s);
      ++a;
      continue;
    }
    size_t b = a;
    while (b < items.size() && items[b].i >= 0 && items[b].key == items[a].key) ++b;
    std::vector<StepSegment> segs;
    for (size_t t = a; t < b && st == LQ_OK; ++t) {
      const int k = items[t].k, i = items[t].i;
      if (k == 1) {
        const int nb[3] = {(i + nc - 1) % nc, i, (i + 1) % nc};
        for (int j : nb)
          if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(s, up[j], 0), "pipeline wait");
      }
      segs.push_back({f[(k - 1) % 2], f[k % 2], sb[i], sb[i + 1]});
    }
    const int t0 = tr.open("step", items[a].i, items[a].k, s);
    if (st == LQ_OK)
      st = stout_step_segments(segs.data(), (int)segs.size(), g, prec, rho, dirs_mask, reproject, tc, s);
    tr.close(t0, s);
    for (size_t t = a + 1; t < b; ++t) tr.alias("step", items[t].i, items[t].k, t0);
    for (size_t t = a; t < b && st == LQ_OK; ++t)
      if (items[t].k == n_steps) {
        st = cuda_check(cudaEventRecord(fin[items[t].i], s), "pipeline final event");
        done_order.push_back(items[t].i);
      }
    a = b;
  }
  void* result = f[n_steps % 2];
  for (int i : done_order) {
    if (st != LQ_OK) break;
    const size_t off = (size_t)sb[i] * site_bytes, len = (size_t)(sb[i + 1] - sb[i]) * site_bytes;
    st = cuda_check(cudaStreamWaitEvent(ps.downx, fin[i], 0), "pipeline wait");
    int t = tr.open("to_aos", i, n_steps, ps.downx);
    if (st == LQ_OK) st = transpose_range(result, stage, g, LQ_LINKS, prec, false, sb[i], sb[i + 1], ps.downx);
    tr.close(t, ps.downx);
    if (st == LQ_OK) st = cuda_check(cudaEventRecord(out_ready[i], ps.downx), "pipeline transpose event");
    if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.down, out_ready[i], 0), "pipeline wait");
    t = tr.open("d2h", i, n_steps, ps.down);
    if (st == LQ_OK)
      st = cuda_check(cudaMemcpyAsync((char*)host_out + off, (const char*)stage + off, len, cudaMemcpyDeviceToHost,
                                      ps.down),
                      "lq_stout_smear_host download");
    tr.close(t, ps.down);
  }
  // the plaquette right after the last step; its two sums are read back on
  // the download stream behind the slab copies (a read-back on s would wait
  // for the copy engine all the same, and hold up the end of the call)
  double* dev_sums = nullptr;
  double sums[2] = {0.0, 0.0};
  if (st == LQ_OK && plaq_out) {
    lq_field tmp;
    tmp.geom = g;
    tmp.kind = LQ_LINKS;
    tmp.prec = prec;
    tmp.ptr = result;
    tmp.bytes = bytes;
    tmp.owned = false;
    st = scratch_alloc((void**)&dev_sums, 2 * sizeof(double), s, "lq_stout_smear_host plaquette");
    const int t = tr.open("plaq", -1, n_steps, s);
    if (st == LQ_OK) st = plaquette_sums_device(&tmp, dev_sums, s);
    tr.close(t, s);
    if (st == LQ_OK) st = cuda_check(cudaEventRecord(plaq_ready, s), "pipeline plaquette event");
    if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.down, plaq_ready, 0), "pipeline wait");
    if (st == LQ_OK)
      st = cuda_check(cudaMemcpyAsync(sums, dev_sums, sizeof(sums), cudaMemcpyDeviceToHost, ps.down),
                      "lq_stout_smear_host plaquette read-back");
  }
  // the scratch goes back to the pool in s's order, after the downloads; on
  // an error the side streams may still hold work that s never waited for
  lq_status st2 = cuda_check(cudaEventRecord(done, ps.down), "pipeline end");
  if (st2 == LQ_OK) st2 = cuda_check(cudaStreamWaitEvent(s, done, 0), "pipeline end");
  if (st != LQ_OK || st2 != LQ_OK) {
    for (cudaStream_t q : {ps.up, ps.upx, ps.down, ps.downx}) cudaStreamSynchronize(q);
  }
  for (void* p : {f[0], f[1], stage, (void*)dev_sums})
    if (p) scratch_free(p, s);
  const lq_status st3 = cuda_check(cudaStreamSynchronize(s), "lq_stout_smear_host sync");
  if (st == LQ_OK && st2 == LQ_OK && st3 == LQ_OK && plaq_out) plaquette_from_sums(sums, V, plaq_out);
  if (st == LQ_OK && st2 == LQ_OK && st3 == LQ_OK) tr.write();
  if (st != LQ_OK) return st;
  return st2 != LQ_OK ? st2 : st3;
}
