// JIT-compiled expression programs.
//
// Winter, "Accelerating QDP++ using GPUs", Sec. 4.1 compiles one CUDA kernel
// per QDP++ expression at run time and keeps it loaded for the life of the
// process; Sec. 8 proposes keeping the compiled code across runs.  Here a
// flattened program (lq_op list) becomes straight-line CUDA C -- every
// register a named local, every kind and shift a compile-time constant --
// compiled by NVRTC for sm_103a into a cubin, cached in memory per program
// and optionally on disk, and launched through driver entry points.  The
// arithmetic is the interpreter's (su3.cuh, expr_ops.cuh, embedded as the
// prelude), so results are bit-identical to lq_expr_eval.
//
// NVRTC is loaded with dlopen on first use and the driver API is reached
// through cudaGetDriverEntryPointByVersion, so the library has no link-time
// dependency on either.
#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lq_internal.h"
#include "reduce.cuh"

namespace lq {

static const char kJitPrelude[] =
#include "jit_prelude.inc"
    ;

lq_status expr_validate(const lq_field* out, const lq_op* prog, int n_ops, const lq_field* const* operands,
                        int n_operands, bool reduce, const char* who);

// ---- NVRTC and driver entry points ------------------------------------------
struct NvrtcApi {
  bool tried = false, ok = false;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};
struct DriverApi {
  bool tried = false, ok = false;
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleGetFunction) get = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
  decltype(&cuModuleUnload) unload = nullptr;
};

static std::mutex g_jit_mu;
static NvrtcApi g_nvrtc;
static DriverApi g_drv;

static bool load_nvrtc() {  // caller holds g_jit_mu
  if (g_nvrtc.tried) return g_nvrtc.ok;
  g_nvrtc.tried = true;
  const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                         "/usr/local/cuda/lib64/libnvrtc.so"};
  void* h = nullptr;
  for (const char* n : names)
    if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) return false;
#define LQ_SYM(field, name) g_nvrtc.field = reinterpret_cast<decltype(g_nvrtc.field)>(dlsym(h, name))
  LQ_SYM(create, "nvrtcCreateProgram");
  LQ_SYM(compile, "nvrtcCompileProgram");
  LQ_SYM(cubin_size, "nvrtcGetCUBINSize");
  LQ_SYM(cubin, "nvrtcGetCUBIN");
  LQ_SYM(log_size, "nvrtcGetProgramLogSize");
  LQ_SYM(log, "nvrtcGetProgramLog");
  LQ_SYM(destroy, "nvrtcDestroyProgram");
#undef LQ_SYM
  g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.cubin_size && g_nvrtc.cubin && g_nvrtc.log_size &&
               g_nvrtc.log && g_nvrtc.destroy;
  return g_nvrtc.ok;
}

static bool load_driver() {  // caller holds g_jit_mu
  if (g_drv.tried) return g_drv.ok;
  g_drv.tried = true;
  cudaDriverEntryPointQueryResult q;
#define LQ_DRV(field, name)                                                                              \
  if (cudaGetDriverEntryPointByVersion(name, reinterpret_cast<void**>(&g_drv.field), 12000, cudaEnableDefault, \
                                       &q) != cudaSuccess ||                                            \
      q != cudaDriverEntryPointSuccess)                                                                 \
    g_drv.field = nullptr;
  LQ_DRV(load, "cuModuleLoadData")
  LQ_DRV(get, "cuModuleGetFunction")
  LQ_DRV(launch, "cuLaunchKernel")
  LQ_DRV(unload, "cuModuleUnload")
#undef LQ_DRV
  cudaGetLastError();
  g_drv.ok = g_drv.load && g_drv.get && g_drv.launch && g_drv.unload;
  return g_drv.ok;
}

// ---- caches ---------------------------------------------------------------------
struct JitModule {
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
};
struct JitEntry {
  std::vector<char> cubin;
  std::map<int, JitModule> per_device;
};
static std::map<std::string, JitEntry>& jit_cache() {
  static std::map<std::string, JitEntry> m;
  return m;
}
static std::string g_cache_dir;
static long long g_stats[4] = {0, 0, 0, 0};  // NVRTC compiles, memory hits, disk hits, module loads

static void release_jit() {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  for (auto& kv : jit_cache())
    for (auto& dm : kv.second.per_device)
      if (dm.second.mod && g_drv.unload) g_drv.unload(dm.second.mod);
  jit_cache().clear();
}

static unsigned long long fnv1a(const std::string& s) {
  unsigned long long h = 1469598103934665603ull;
  for (unsigned char ch : s) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

// ---- code generation ------------------------------------------------------------
static std::string hexf(double v) {
  char b[64];
  snprintf(b, sizeof(b), "%a", v);
  return b;
}

static std::string gen_source(const lq_field* out, const lq_op* prog, int n_ops, const lq_field* const* operands,
                              bool reduce) {
  const int prec = operands[0]->prec;
  std::string src(kJitPrelude);
  src += "\nnamespace lq {\nstruct JitArgs {\n  const void* op[8];\n  void* out;\n  double* parts;\n  GeomArgs g;\n};\n}\n";
  src += "extern \"C\" __global__ void __launch_bounds__(256) lq_jit_expr(lq::JitArgs a) {\n";
  src += "  using namespace lq;\n";
  src += std::string("  typedef ") + (prec == LQ_F64 ? "double" : "float") + " Real;\n";
  src += "  const long long V = a.g.V;\n  double acc[2] = {0.0, 0.0};\n";
  src += "  for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < V;\n"
         "       sl += (long long)gridDim.x * blockDim.x) {\n";
  src += "    const int s = (int)sl;\n    int c[4];\n    site_coords(a.g, s, c);\n";
  src += "    M3<Real> r0, r1, r2, r3, r4, r5, r6, r7;\n";
  int res = 0;
  char line[512];
  for (int i = 0; i < n_ops; ++i) {
    const lq_op& o = prog[i];
    switch (o.code) {
      case LQ_OP_LOAD: {
        std::string site = "s";
        if (o.sign > 0) {
          snprintf(line, sizeof(line), "nb_fwd(a.g, s, c[%d], %d)", o.mu, o.mu);
          site = line;
        } else if (o.sign < 0) {
          snprintf(line, sizeof(line), "nb_bwd(a.g, s, c[%d], %d)", o.mu, o.mu);
          site = line;
        }
        const int kind = operands[o.a]->kind;
        snprintf(line, sizeof(line), "    r%d = load_operand<Real>(a.op[%d], %d, %d, V, %s);\n", o.dst, o.a, kind,
                 kind == LQ_LINKS ? o.dir : 0, site.c_str());
        break;
      }
      case LQ_OP_ADJ: snprintf(line, sizeof(line), "    r%d = m_adj(r%d);\n", o.dst, o.a); break;
      case LQ_OP_MUL: snprintf(line, sizeof(line), "    r%d = mul_nn(r%d, r%d);\n", o.dst, o.a, o.b); break;
      case LQ_OP_ADD: snprintf(line, sizeof(line), "    r%d = m_add(r%d, r%d);\n", o.dst, o.a, o.b); break;
      case LQ_OP_SUB: snprintf(line, sizeof(line), "    r%d = m_sub(r%d, r%d);\n", o.dst, o.a, o.b); break;
      case LQ_OP_SCALE:
        snprintf(line, sizeof(line), "    r%d = m_scale(r%d, mkc<Real>((Real)%s, (Real)%s));\n", o.dst, o.a,
                 hexf(o.re).c_str(), hexf(o.im).c_str());
        break;
      case LQ_OP_TRACE:
        snprintf(line, sizeof(line),
                 "    { const cx<Real> t = m_trace(r%d); M3<Real> m; m_zero(m); m.e[0] = m.e[4] = m.e[8] = t; "
                 "r%d = m; }\n",
                 o.a, o.dst);
        break;
      case LQ_OP_RETR:
        snprintf(line, sizeof(line),
                 "    { const cx<Real> t = m_trace(r%d); M3<Real> m; m_zero(m); m.e[0] = m.e[4] = m.e[8] = "
                 "mkc<Real>(t.re, 0); r%d = m; }\n",
                 o.a, o.dst);
        break;
      default:
        res = o.a;
        line[0] = 0;
        break;
    }
    src += line;
  }
  if (out) {
    snprintf(line, sizeof(line), "    store_result<Real>(a.out, %d, V, s, r%d);\n", out->kind, res);
    src += line;
  }
  if (reduce) {
    snprintf(line, sizeof(line),
             "    { const cx<Real> t = m_trace(r%d); acc[0] += (double)t.re; acc[1] += (double)t.im; }\n", res);
    src += line;
  }
  src += "  }\n";
  if (reduce) src += "  block_sum_store<2>(acc, a.parts + 2 * blockIdx.x);\n";
  src += "}\n";
  return src;
}

static bool read_file(const std::string& path, std::vector<char>& data) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  fseek(f, 0, SEEK_END);
  long n = ftell(f);
  fseek(f, 0, SEEK_SET);
  data.resize(n > 0 ? (size_t)n : 0);
  const bool ok = n > 0 && fread(data.data(), 1, (size_t)n, f) == (size_t)n;
  fclose(f);
  return ok;
}
static void write_file(const std::string& path, const char* data, size_t n) {
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(data, 1, n, f) == n;
  fclose(f);
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

// The cubin of `src`: from memory, the disk cache, or NVRTC.  Holds g_jit_mu.
static lq_status get_cubin(const std::string& src, JitEntry** out) {
  auto it = jit_cache().find(src);
  if (it != jit_cache().end()) {
    ++g_stats[1];
    *out = &it->second;
    return LQ_OK;
  }
  JitEntry e;
  char hash[32];
  snprintf(hash, sizeof(hash), "%016llx", fnv1a(src));
  const std::string base = g_cache_dir.empty() ? std::string() : g_cache_dir + "/lqjit_" + hash;
  if (!base.empty()) {
    std::vector<char> stored_src;
    if (read_file(base + ".cu", stored_src) && stored_src.size() == src.size() &&
        memcmp(stored_src.data(), src.data(), src.size()) == 0 && read_file(base + ".cubin", e.cubin)) {
      ++g_stats[2];
      *out = &jit_cache().emplace(src, std::move(e)).first->second;
      return LQ_OK;
    }
  }
  if (!load_nvrtc()) {
    set_error("lq_expr_jit: NVRTC (libnvrtc.so) could not be loaded");
    return LQ_ERR_UNSUPPORTED;
  }
  nvrtcProgram p = nullptr;
  if (g_nvrtc.create(&p, src.c_str(), "lq_jit_expr.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    set_error("lq_expr_jit: nvrtcCreateProgram failed");
    return LQ_ERR_CUDA;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=true", "-lineinfo"};
  const nvrtcResult rc = g_nvrtc.compile(p, 4, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    g_nvrtc.log_size(p, &n);
    std::string log(n, '\0');
    if (n) g_nvrtc.log(p, &log[0]);
    g_nvrtc.destroy(&p);
    set_error("lq_expr_jit: NVRTC compilation failed: %.400s", log.c_str());
    return LQ_ERR_CUDA;
  }
  size_t n = 0;
  g_nvrtc.cubin_size(p, &n);
  e.cubin.resize(n);
  g_nvrtc.cubin(p, e.cubin.data());
  g_nvrtc.destroy(&p);
  ++g_stats[0];
  if (!base.empty()) {
    write_file(base + ".cu", src.data(), src.size());
    write_file(base + ".cubin", e.cubin.data(), e.cubin.size());
  }
  *out = &jit_cache().emplace(src, std::move(e)).first->second;
  return LQ_OK;
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_expr_jit_prepare(const lq_field* out_or_null, const lq_op* prog, int n_ops,
                                         const lq_field* const* operands, int n_operands, int reduce) {
  clear_error();
  lq_status st = expr_validate(out_or_null, prog, n_ops, operands, n_operands, reduce != 0, "lq_expr_jit_prepare");
  if (st != LQ_OK) return st;
  const std::string src = gen_source(out_or_null, prog, n_ops, operands, reduce != 0);
  register_cache_release(release_jit);
  std::lock_guard<std::mutex> lk(g_jit_mu);
  JitEntry* e = nullptr;
  return get_cubin(src, &e);
}

extern "C" lq_status lq_expr_eval_jit(lq_field* out, const lq_op* prog, int n_ops, const lq_field* const* operands,
                                      int n_operands, double* reduce_out, void* stream) {
  clear_error();
  lq_status st = expr_validate(out, prog, n_ops, operands, n_operands, reduce_out != nullptr, "lq_expr_eval_jit");
  if (st != LQ_OK) return st;
  const std::string src = gen_source(out, prog, n_ops, operands, reduce_out != nullptr);
  register_cache_release(release_jit);
  cudaStream_t s = as_stream(stream);
  CUfunction fn = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    JitEntry* e = nullptr;
    if ((st = get_cubin(src, &e)) != LQ_OK) return st;
    const int dev = current_device();
    auto dm = e->per_device.find(dev);
    if (dm == e->per_device.end()) {
      if ((st = cuda_check(cudaFree(nullptr), "lq_expr_eval_jit context"))) return st;  // primary context current
      if (!load_driver()) {
        set_error("lq_expr_eval_jit: driver entry points unavailable");
        return LQ_ERR_UNSUPPORTED;
      }
      JitModule m;
      if (g_drv.load(&m.mod, e->cubin.data()) != CUDA_SUCCESS || g_drv.get(&m.fn, m.mod, "lq_jit_expr") != CUDA_SUCCESS) {
        if (m.mod) g_drv.unload(m.mod);
        set_error("lq_expr_eval_jit: loading the compiled module failed");
        return LQ_ERR_CUDA;
      }
      ++g_stats[3];
      dm = e->per_device.emplace(dev, m).first;
    }
    fn = dm->second.fn;
  }
  struct JitArgsHost {
    const void* op[8];
    void* out;
    double* parts;
    GeomArgs g;
  } args;
  memset(&args, 0, sizeof(args));
  for (int k = 0; k < n_operands; ++k) args.op[k] = operands[k]->ptr;
  args.out = out ? out->ptr : nullptr;
  args.g = geom_args(operands[0]->geom);
  const int grid = reduce_grid(args.g.V);
  double* scratch = nullptr;
  if (reduce_out) {
    if ((st = scratch_alloc((void**)&scratch, sizeof(double) * 2 * (grid + 1), s, "lq_expr_eval_jit"))) return st;
    args.parts = scratch;
  }
  void* params[] = {&args};
  const CUresult lr = g_drv.launch(fn, (unsigned)grid, 1, 1, kReduceThreads, 1, 1, 0, (CUstream)s, params, nullptr);
  st = lr == CUDA_SUCCESS ? LQ_OK : LQ_ERR_CUDA;
  if (st != LQ_OK) set_error("lq_expr_eval_jit: cuLaunchKernel failed (%d)", (int)lr);
  if (!reduce_out) return st;
  if (st == LQ_OK) {
    k_reduce_partials<2><<<1, kReduceThreads, 0, s>>>(scratch, grid, scratch + 2 * grid);
    st = launch_check("lq_expr_eval_jit reduce");
  }
  double host[2] = {0, 0};
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpyAsync(host, scratch + 2 * grid, sizeof(host), cudaMemcpyDeviceToHost, s),
                    "lq_expr_eval_jit copy");
  scratch_free(scratch, s);
  lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_expr_eval_jit sync");
  if (st == LQ_OK) st = st2;
  if (st == LQ_OK) {
    reduce_out[0] = host[0];
    reduce_out[1] = host[1];
  }
  return st;
}

extern "C" lq_status lq_jit_cache_dir(const char* path) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_jit_mu);
  g_cache_dir = path ? path : "";
  return LQ_OK;
}

extern "C" lq_status lq_jit_stats(long long out[4]) {
  clear_error();
  if (!out) {
    set_error("lq_jit_stats: NULL output");
    return LQ_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_jit_mu);
  for (int i = 0; i < 4; ++i) out[i] = g_stats[i];
  return LQ_OK;
}
