// Stout smearing of links held in host memory, with the host<->device
// transfers pipelined against the smearing.  The lattice is cut into slabs of
// whole t-slices (contiguous site ranges in the lexicographic order, so a slab
// is one contiguous piece of the host AoS array and of every SoA plane).
//   upload stream:   per slab, H2D copy into an AoS staging buffer, then the
//                    AoS -> SoA transpose of that slab; event up[i].
//   compute stream:  step 1 of slab i waits for up[i-1], up[i], up[i+1] (the
//                    staples reach one t-slice into each neighbour); steps
//                    2..n follow in stream order, slab by slab; after the
//                    last step of slab i, event fin[i].
//   download stream: per slab, waits for fin[i], transposes the slab back into
//                    the staging buffer and copies it to the host.
// Step k of a slab reads field (k-1)%2 and writes field k%2; stream order
// runs step k of every slab before step k+1 of any, which covers both the
// reads of step k+1 and the overwrite of field (k+1)%2 by step k+1.
// (Winter, "Accelerating QDP++ using GPUs", Sec. 4.3 moves whole fields
// between host and device on demand; here the device layout stays fixed and
// the transfers run behind the arithmetic.)
#include <vector>

#include "lq_internal.h"

using namespace lq;

namespace {

struct Streams {
  cudaStream_t up = nullptr, down = nullptr;
  std::vector<cudaEvent_t> ev;
  ~Streams() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
  }
  lq_status make(int n_events) {
    lq_status st = cuda_check(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking), "upload stream");
    if (st == LQ_OK) st = cuda_check(cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking), "download stream");
    for (int i = 0; i < n_events && st == LQ_OK; ++i) {
      cudaEvent_t e;
      st = cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "pipeline event");
      if (st == LQ_OK) ev.push_back(e);
    }
    return st;
  }
};

int slab_count(int Lt, int n_chunks) {
  int nc = n_chunks > 0 ? n_chunks : 8;
  return nc > Lt ? Lt : nc;
}

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
  if ((st = ps.make(2 * nc + 2)) != LQ_OK) return st;
  cudaEvent_t* up = ps.ev.data();
  cudaEvent_t* fin = ps.ev.data() + nc;
  cudaEvent_t start = ps.ev[2 * nc], done = ps.ev[2 * nc + 1];

  void* f[2] = {nullptr, nullptr};
  void* stage = nullptr;
  if (st == LQ_OK) st = scratch_alloc(&f[0], bytes, s, "lq_stout_smear_host field");
  if (st == LQ_OK && n_steps > 0) st = scratch_alloc(&f[1], bytes, s, "lq_stout_smear_host work field");
  if (st == LQ_OK) st = scratch_alloc(&stage, bytes, s, "lq_stout_smear_host staging");
  // the side streams start after the allocations (and all earlier work) on s
  if (st == LQ_OK) st = cuda_check(cudaEventRecord(start, s), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.up, start, 0), "pipeline start");
  if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(ps.down, start, 0), "pipeline start");

  const size_t site_bytes = 4 * 9 * eb;
  const size_t plane = (size_t)V * eb;
  for (int i = 0; i < nc && st == LQ_OK; ++i) {
    const size_t off = (size_t)sb[i] * site_bytes, len = (size_t)(sb[i + 1] - sb[i]) * site_bytes;
    st = cuda_check(cudaMemcpyAsync((char*)stage + off, (const char*)host_in + off, len, cudaMemcpyHostToDevice,
                                    ps.up),
                    "lq_stout_smear_host upload");
    if (st == LQ_OK) st = transpose_range(stage, f[0], g, LQ_LINKS, prec, true, sb[i], sb[i + 1], ps.up);
    // links outside dirs are never written: the work field needs them too
    for (int mu = 0; mu < 4 && st == LQ_OK && n_steps > 0; ++mu)
      if (!((dirs_mask >> mu) & 1u))
        for (int c = 0; c < 9 && st == LQ_OK; ++c) {
          const size_t po = (size_t)(mu * 9 + c) * plane + (size_t)sb[i] * eb;
          st = cuda_check(cudaMemcpyAsync((char*)f[1] + po, (const char*)f[0] + po, (size_t)(sb[i + 1] - sb[i]) * eb,
                                          cudaMemcpyDeviceToDevice, ps.up),
                          "lq_stout_smear_host pass-through copy");
        }
    if (st == LQ_OK) st = cuda_check(cudaEventRecord(up[i], ps.up), "pipeline upload event");
  }

  // step 1 in the order 1, 2, ..., nc-1, 0: each slab as soon as it and its
  // neighbours are resident (slab 0 borders slab nc-1 periodically)
  std::vector<int> order;
  for (int i = 1; i < nc; ++i) order.push_back(i);
  order.push_back(0);
  if (n_steps == 0)
    for (int i = 0; i < nc && st == LQ_OK; ++i) st = cuda_check(cudaStreamWaitEvent(s, up[i], 0), "pipeline wait");
  for (int k = 1; k <= n_steps && st == LQ_OK; ++k) {
    const void* in = f[(k - 1) % 2];
    void* out = f[k % 2];
    for (int i : order) {
      if (k == 1) {
        const int nb[3] = {(i + nc - 1) % nc, i, (i + 1) % nc};
        for (int j : nb)
          if (st == LQ_OK) st = cuda_check(cudaStreamWaitEvent(s, up[j], 0), "pipeline wait");
      }
      if (st == LQ_OK) st = stout_step_range(in, out, g, prec, rho, dirs_mask, reproject, tc, sb[i], sb[i + 1], s);
      if (st == LQ_OK && k == n_steps) st = cuda_check(cudaEventRecord(fin[i], s), "pipeline final event");
      if (st != LQ_OK) break;
    }
  }
  void* result = f[n_steps % 2];
  if (n_steps == 0 && st == LQ_OK)
    for (int i = 0; i < nc && st == LQ_OK; ++i) st = cuda_check(cudaEventRecord(fin[i], s), "pipeline final event");
  for (int i : order) {
    if (st != LQ_OK) break;
    const size_t off = (size_t)sb[i] * site_bytes, len = (size_t)(sb[i + 1] - sb[i]) * site_bytes;
    st = cuda_check(cudaStreamWaitEvent(ps.down, fin[i], 0), "pipeline wait");
    if (st == LQ_OK) st = transpose_range(result, stage, g, LQ_LINKS, prec, false, sb[i], sb[i + 1], ps.down);
    if (st == LQ_OK)
      st = cuda_check(cudaMemcpyAsync((char*)host_out + off, (const char*)stage + off, len, cudaMemcpyDeviceToHost,
                                      ps.down),
                      "lq_stout_smear_host download");
  }
  if (st == LQ_OK && plaq_out) {
    lq_field tmp;
    tmp.geom = g;
    tmp.kind = LQ_LINKS;
    tmp.prec = prec;
    tmp.ptr = result;
    tmp.bytes = bytes;
    tmp.owned = false;
    st = lq_plaquette(&tmp, plaq_out, stream);
  }
  // the scratch goes back to the pool in s's order, after the downloads; on
  // an error the side streams may still hold work that s never waited for
  lq_status st2 = cuda_check(cudaEventRecord(done, ps.down), "pipeline end");
  if (st2 == LQ_OK) st2 = cuda_check(cudaStreamWaitEvent(s, done, 0), "pipeline end");
  if (st != LQ_OK || st2 != LQ_OK) {
    cudaStreamSynchronize(ps.up);
    cudaStreamSynchronize(ps.down);
  }
  for (void* p : {f[0], f[1], stage})
    if (p) scratch_free(p, s);
  const lq_status st3 = cuda_check(cudaStreamSynchronize(s), "lq_stout_smear_host sync");
  if (st != LQ_OK) return st;
  return st2 != LQ_OK ? st2 : st3;
}
