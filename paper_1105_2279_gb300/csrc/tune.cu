// Auto-tuner cache: the best (block size N_threads, sites per thread N_site,
// kernel variant) per (kernel, precision, dims, smeared directions, device),
// found by timing the candidates once and kept for later runs (the tuning
// step that Winter, "Accelerating QDP++ using GPUs", Secs. 4.4 and 8,
// proposes to run before production).  Text cache, one entry per line:
//   <kernel> <device name with '_' for ' '> <prec> <Lx> <Ly> <Lz> <Lt> <dirs> <block> <nsite> <variant>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "lq_internal.h"

namespace lq {

static std::mutex g_tune_mu;
static bool g_tune_on = false;
static std::string g_tune_path;
static std::map<std::string, TuneChoice>& tune_map() {
  static std::map<std::string, TuneChoice> m;
  return m;
}

static std::string device_name() {
  cudaDeviceProp p;
  std::memset(&p, 0, sizeof(p));
  if (cudaGetDeviceProperties(&p, current_device()) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n(p.name);
  for (auto& ch : n)
    if (ch == ' ') ch = '_';
  return n;
}

static std::string make_key(const char* kernel, const std::string& dev, int prec, const int d[4], unsigned dirs) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s %s %d %d %d %d %d %u", kernel, dev.c_str(), prec, d[0], d[1], d[2], d[3], dirs);
  return buf;
}

static void save_locked() {
  if (g_tune_path.empty()) return;
  FILE* f = fopen(g_tune_path.c_str(), "w");
  if (!f) return;
  for (auto& kv : tune_map())
    fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.block, kv.second.nsite, kv.second.variant);
  fclose(f);
}

bool tune_enabled() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune_on;
}

bool tune_get(const char* kernel, int prec, const int dims[4], unsigned dirs, TuneChoice* out) {
  std::string k = make_key(kernel, device_name(), prec, dims, dirs);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = tune_map().find(k);
  if (it == tune_map().end()) return false;
  *out = it->second;
  return true;
}

void tune_put(const char* kernel, int prec, const int dims[4], unsigned dirs, const TuneChoice& c) {
  std::string k = make_key(kernel, device_name(), prec, dims, dirs);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_map()[k] = c;
  save_locked();
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_tune(const char* cache_path) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_on = true;
  g_tune_path = cache_path ? cache_path : "";
  if (g_tune_path.empty()) return LQ_OK;
  FILE* f = fopen(g_tune_path.c_str(), "r");
  if (!f) return LQ_OK;  // created on the first new entry
  char kernel[64], dev[160];
  int prec, d0, d1, d2, d3, b, ns, var;
  unsigned dirs;
  while (fscanf(f, "%63s %159s %d %d %d %d %d %u %d %d %d", kernel, dev, &prec, &d0, &d1, &d2, &d3, &dirs, &b, &ns,
                &var) == 11) {
    const int d[4] = {d0, d1, d2, d3};
    TuneChoice c;
    c.block = b;
    c.nsite = ns;
    c.variant = var;
    if (b > 0 && b <= 1024 && ns > 0 && ns <= 64) tune_map()[make_key(kernel, dev, prec, d, dirs)] = c;
  }
  fclose(f);
  return LQ_OK;
}

extern "C" lq_status lq_tune_lookup(int prec, const int dims[4], unsigned dirs_mask, int* block,
                                    int* sites_per_thread, int* variant) {
  clear_error();
  if (!dims) {
    set_error("lq_tune_lookup: NULL dims");
    return LQ_ERR_ARG;
  }
  TuneChoice c;
  if (!tune_get("stout", prec, dims, dirs_mask, &c)) {
    set_error("lq_tune_lookup: no entry");
    return LQ_ERR_ARG;
  }
  if (block) *block = c.block;
  if (sites_per_thread) *sites_per_thread = c.nsite;
  if (variant) *variant = c.variant;
  return LQ_OK;
}
