// Nearest-neighbour shift and the fused per-site expression evaluator.
//
// Winter, "Accelerating QDP++ using GPUs", Sec. 4.2 evaluates one expression
// per kernel from a flattened expression tree, with shift served by device
// site tables; Listing 1 (Sec. 6) fixes the operations (shift FORWARD /
// BACKWARD, adj, products, sums, scalar multiples).  Here the flattened form
// is a short register program interpreted per site, and neighbours come from
// index arithmetic instead of tables.
#include <cstring>

#include "expr_ops.cuh"
#include "lq_internal.h"
#include "reduce.cuh"
#include "stout_core.cuh"

static_assert(lq::kKindLinks == LQ_LINKS && lq::kKindMatrix == LQ_COLOR_MATRIX && lq::kKindVector == LQ_COLOR_VECTOR &&
                  lq::kKindComplex == LQ_COMPLEX && lq::kKindReal == LQ_REAL,
              "field kind numbering");

namespace lq {

// ---- shift -----------------------------------------------------------------
template <typename E>
__global__ void k_shift(const E* __restrict__ in, E* __restrict__ out, GeomArgs g, int planes, int mu, int sign) {
  const long long V = g.V;
  for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < V;
       sl += (long long)gridDim.x * blockDim.x) {
    const int s = (int)sl;
    int c[4];
    site_coords(g, s, c);
    const int cm = coord_of(c, mu);
    const int src = sign > 0 ? nb_fwd(g, s, cm, mu) : nb_bwd(g, s, cm, mu);
    for (int p = 0; p < planes; ++p) out[(long long)p * V + s] = __ldg(in + (long long)p * V + src);
  }
}

// ---- expression programs -----------------------------------------------------
struct DevOp {
  signed char code, dst, a, b, dir, mu, sign, pad;
};
struct DevProg {
  int n_ops;
  int n_operands;
  DevOp ops[LQ_EXPR_MAX_OPS];
  double sre[LQ_EXPR_MAX_OPS], sim[LQ_EXPR_MAX_OPS];
  const void* operand[LQ_EXPR_MAX_OPERANDS];
  int operand_kind[LQ_EXPR_MAX_OPERANDS];
};

template <typename R>
__global__ void __launch_bounds__(kReduceThreads) k_expr(DevProg prog, GeomArgs g, void* out, int out_kind,
                                                         double* parts) {
  const long long V = g.V;
  M3<R> reg[LQ_EXPR_MAX_REGS];
  double acc[2] = {0.0, 0.0};
  for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < V;
       sl += (long long)gridDim.x * blockDim.x) {
    const int s = (int)sl;
    int c[4];
    site_coords(g, s, c);
    int res = 0;
    for (int i = 0; i < prog.n_ops; ++i) {
      const DevOp op = prog.ops[i];
      switch (op.code) {
        case LQ_OP_LOAD: {
          int site = s;
          if (op.sign > 0) site = nb_fwd(g, s, coord_of(c, op.mu), op.mu);
          if (op.sign < 0) site = nb_bwd(g, s, coord_of(c, op.mu), op.mu);
          reg[op.dst] = load_operand<R>(prog.operand[op.a], prog.operand_kind[op.a], op.dir, V, site);
          break;
        }
        case LQ_OP_ADJ: reg[op.dst] = m_adj(reg[op.a]); break;
        case LQ_OP_MUL: reg[op.dst] = mul_nn(reg[op.a], reg[op.b]); break;
        case LQ_OP_ADD: reg[op.dst] = m_add(reg[op.a], reg[op.b]); break;
        case LQ_OP_SUB: reg[op.dst] = m_sub(reg[op.a], reg[op.b]); break;
        case LQ_OP_SCALE: reg[op.dst] = m_scale(reg[op.a], mkc<R>((R)prog.sre[i], (R)prog.sim[i])); break;
        case LQ_OP_TRACE: {
          const cx<R> t = m_trace(reg[op.a]);
          M3<R> m;
          m_zero(m);
          m.e[0] = m.e[4] = m.e[8] = t;
          reg[op.dst] = m;
          break;
        }
        case LQ_OP_RETR: {
          const cx<R> t = m_trace(reg[op.a]);
          M3<R> m;
          m_zero(m);
          m.e[0] = m.e[4] = m.e[8] = mkc<R>(t.re, 0);
          reg[op.dst] = m;
          break;
        }
        default: res = op.a; break;  // LQ_OP_STORE
      }
    }
    if (out) store_result<R>(out, out_kind, V, s, reg[res]);
    if (parts) {
      const cx<R> t = m_trace(reg[res]);
      acc[0] += (double)t.re;
      acc[1] += (double)t.im;
    }
  }
  if (parts) block_sum_store<2>(acc, parts + 2 * blockIdx.x);
}

}  // namespace lq

using namespace lq;

extern "C" lq_status lq_shift(lq_field* out, const lq_field* in, int mu, int sign, void* stream) {
  clear_error();
  if (!out || !in) {
    set_error("lq_shift: NULL field");
    return LQ_ERR_ARG;
  }
  if (mu < 0 || mu > 3 || (sign != 1 && sign != -1)) {
    set_error("lq_shift: mu must be in [0,3] and sign +1 or -1 (got %d, %d)", mu, sign);
    return LQ_ERR_ARG;
  }
  if (!same_geom(out->geom, in->geom) || out->kind != in->kind || out->prec != in->prec) {
    set_error("lq_shift: in and out differ in geometry, kind or precision");
    return LQ_ERR_GEOM;
  }
  if (out->ptr == in->ptr) {
    set_error("lq_shift: in and out must not alias");
    return LQ_ERR_ARG;
  }
  cudaStream_t s = as_stream(stream);
  const GeomArgs g = geom_args(in->geom);
  const int planes = ndir_of(in->kind) * ncomp_of(in->kind);
  const int grid = (int)std::min<long long>((g.V + 255) / 256, (long long)device_sm_count() * 8);
  const size_t eb = elem_bytes(in->kind, in->prec);
  if (eb == 16)
    k_shift<double2><<<grid, 256, 0, s>>>((const double2*)in->ptr, (double2*)out->ptr, g, planes, mu, sign);
  else if (eb == 8)
    k_shift<float2><<<grid, 256, 0, s>>>((const float2*)in->ptr, (float2*)out->ptr, g, planes, mu, sign);
  else
    k_shift<float><<<grid, 256, 0, s>>>((const float*)in->ptr, (float*)out->ptr, g, planes, mu, sign);
  return launch_check("lq_shift");
}

namespace lq {

// Checks a program and its fields for lq_expr_eval / lq_expr_eval_jit / lq_expr_jit_prepare.
lq_status expr_validate(const lq_field* out, const lq_op* prog, int n_ops, const lq_field* const* operands,
                        int n_operands, bool reduce, const char* who) {
  if (!prog || n_ops < 1 || n_ops > LQ_EXPR_MAX_OPS || !operands || n_operands < 1 ||
      n_operands > LQ_EXPR_MAX_OPERANDS) {
    set_error("%s: need 1..%d ops and 1..%d operands", who, LQ_EXPR_MAX_OPS, LQ_EXPR_MAX_OPERANDS);
    return LQ_ERR_ARG;
  }
  if (!out && !reduce) {
    set_error("%s: neither an output field nor a reduction was requested", who);
    return LQ_ERR_ARG;
  }
  const lq_field* f0 = operands[0];
  for (int k = 0; k < n_operands; ++k) {
    if (!operands[k]) {
      set_error("%s: operand %d is NULL", who, k);
      return LQ_ERR_ARG;
    }
    if (!same_geom(operands[k]->geom, f0->geom) || operands[k]->prec != f0->prec) {
      set_error("%s: operand %d differs in geometry or precision", who, k);
      return LQ_ERR_GEOM;
    }
    if (operands[k]->kind == LQ_FERMION) {
      set_error("%s: FERMION operands are not supported by the 3x3 register machine", who);
      return LQ_ERR_UNSUPPORTED;
    }
  }
  if (out) {
    if (!same_geom(out->geom, f0->geom) || out->prec != f0->prec || out->kind == LQ_LINKS ||
        out->kind == LQ_FERMION) {
      set_error("%s: output must share geometry/precision and not be LQ_LINKS or LQ_FERMION", who);
      return LQ_ERR_GEOM;
    }
    for (int k = 0; k < n_operands; ++k)
      if (operands[k]->ptr == out->ptr) {
        set_error("%s: output aliases operand %d", who, k);
        return LQ_ERR_ARG;
      }
  }
  for (int i = 0; i < n_ops; ++i) {
    const lq_op& o = prog[i];
    const bool last = (i == n_ops - 1);
    bool ok = o.code >= LQ_OP_LOAD && o.code <= LQ_OP_STORE && (o.code == LQ_OP_STORE) == last;
    const bool uses_a_reg = o.code != LQ_OP_LOAD;
    const bool uses_b = o.code == LQ_OP_MUL || o.code == LQ_OP_ADD || o.code == LQ_OP_SUB;
    if (ok && o.code != LQ_OP_STORE) ok = o.dst >= 0 && o.dst < LQ_EXPR_MAX_REGS;
    if (ok && uses_a_reg) ok = o.a >= 0 && o.a < LQ_EXPR_MAX_REGS;
    if (ok && uses_b) ok = o.b >= 0 && o.b < LQ_EXPR_MAX_REGS;
    if (ok && o.code == LQ_OP_LOAD) {
      ok = o.a >= 0 && o.a < n_operands && o.sign >= -1 && o.sign <= 1 && (o.sign == 0 || (o.mu >= 0 && o.mu <= 3));
      if (ok) ok = operands[o.a]->kind == LQ_LINKS ? (o.dir >= 0 && o.dir < 4) : true;
    }
    if (ok && o.code == LQ_OP_SCALE) ok = o.re == o.re && o.im == o.im;
    if (!ok) {
      set_error("%s: op %d (code %d) is malformed", who, i, o.code);
      return LQ_ERR_ARG;
    }
  }
  return LQ_OK;
}

}  // namespace lq

extern "C" lq_status lq_expr_eval(lq_field* out, const lq_op* prog, int n_ops, const lq_field* const* operands,
                                  int n_operands, double* reduce_out, void* stream) {
  clear_error();
  lq_status st = expr_validate(out, prog, n_ops, operands, n_operands, reduce_out != nullptr, "lq_expr_eval");
  if (st != LQ_OK) return st;
  const lq_field* f0 = operands[0];
  DevProg dp;
  std::memset(&dp, 0, sizeof(dp));
  dp.n_ops = n_ops;
  dp.n_operands = n_operands;
  for (int k = 0; k < n_operands; ++k) {
    dp.operand[k] = operands[k]->ptr;
    dp.operand_kind[k] = operands[k]->kind;
  }
  for (int i = 0; i < n_ops; ++i) {
    const lq_op& o = prog[i];
    const bool uses_b = o.code == LQ_OP_MUL || o.code == LQ_OP_ADD || o.code == LQ_OP_SUB;
    DevOp d;
    d.code = (signed char)o.code;
    d.dst = (signed char)(o.code == LQ_OP_STORE ? 0 : o.dst);
    d.a = (signed char)o.a;
    d.b = (signed char)(uses_b ? o.b : 0);
    d.dir = (signed char)(o.code == LQ_OP_LOAD && operands[o.a]->kind == LQ_LINKS ? o.dir : 0);
    d.mu = (signed char)(o.code == LQ_OP_LOAD ? o.mu : 0);
    d.sign = (signed char)(o.code == LQ_OP_LOAD ? o.sign : 0);
    d.pad = 0;
    dp.ops[i] = d;
    dp.sre[i] = o.re;
    dp.sim[i] = o.im;
  }
  cudaStream_t s = as_stream(stream);
  const GeomArgs g = geom_args(f0->geom);
  const int grid = reduce_grid(g.V);
  void* outp = out ? out->ptr : nullptr;
  const int out_kind = out ? out->kind : LQ_COLOR_MATRIX;
  double* scratch = nullptr;
  if (reduce_out) {
    st = scratch_alloc((void**)&scratch, sizeof(double) * 2 * (grid + 1), s, "lq_expr_eval");
    if (st != LQ_OK) return st;
  }
  if (f0->prec == LQ_F64)
    k_expr<double><<<grid, kReduceThreads, 0, s>>>(dp, g, outp, out_kind, scratch);
  else
    k_expr<float><<<grid, kReduceThreads, 0, s>>>(dp, g, outp, out_kind, scratch);
  st = launch_check("lq_expr_eval");
  if (!reduce_out) return st;
  if (st == LQ_OK) {
    k_reduce_partials<2><<<1, kReduceThreads, 0, s>>>(scratch, grid, scratch + 2 * grid);
    st = launch_check("lq_expr_eval reduce");
  }
  double host[2] = {0, 0};
  if (st == LQ_OK)
    st = cuda_check(cudaMemcpyAsync(host, scratch + 2 * grid, sizeof(host), cudaMemcpyDeviceToHost, s), "lq_expr_eval copy");
  scratch_free(scratch, s);
  lq_status st2 = cuda_check(cudaStreamSynchronize(s), "lq_expr_eval sync");
  if (st == LQ_OK) st = st2;
  if (st == LQ_OK) {
    reduce_out[0] = host[0];
    reduce_out[1] = host[1];
  }
  return st;
}
