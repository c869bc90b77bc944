// Operand loads and result stores of the per-site expression programs,
// shared by the interpreter (expr.cu) and the NVRTC-compiled kernels (jit.cu),
// so both evaluate a program with the same arithmetic.  Compiles under NVRTC.
#pragma once

#include "su3.cuh"

namespace lq {

// field kinds (the values of lq_kind in lqcd.h)
enum { kKindLinks = 0, kKindMatrix = 1, kKindVector = 2, kKindComplex = 3, kKindReal = 4 };

// A LINKS / COLOR_MATRIX operand loads as its matrix (direction `dir` of a
// LINKS field), a COLOR_VECTOR into column 0, COMPLEX / REAL as scalar * 1.
template <typename R>
__device__ __forceinline__ M3<R> load_operand(const void* base, int kind, int dir, long long V, int s) {
  typedef typename vec2<R>::type V2;
  M3<R> m;
  m_zero(m);
  if (kind == kKindLinks || kind == kKindMatrix) {
    m = ld_m3<R>((const V2*)base + (long long)dir * 9 * V + s, V);
  } else if (kind == kKindVector) {
    const V2* p = (const V2*)base + s;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      V2 v = __ldg(p + r * V);
      m.e[3 * r] = mkc<R>(v.x, v.y);
    }
  } else if (kind == kKindComplex) {
    V2 v = __ldg((const V2*)base + s);
    m.e[0] = m.e[4] = m.e[8] = mkc<R>(v.x, v.y);
  } else {
    R v = __ldg((const R*)base + s);
    m.e[0] = m.e[4] = m.e[8] = mkc<R>(v, 0);
  }
  return m;
}

template <typename R>
__device__ __forceinline__ void store_result(void* base, int kind, long long V, int s, const M3<R>& m) {
  typedef typename vec2<R>::type V2;
  if (kind == kKindMatrix) {
    st_m3<R>((V2*)base + s, V, m);
  } else if (kind == kKindVector) {
    V2* p = (V2*)base + s;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      V2 v;
      v.x = m.e[3 * r].re;
      v.y = m.e[3 * r].im;
      p[r * V] = v;
    }
  } else if (kind == kKindComplex) {
    V2 v;
    v.x = m.e[0].re;
    v.y = m.e[0].im;
    ((V2*)base)[s] = v;
  } else {
    ((R*)base)[s] = m.e[0].re;
  }
}

}  // namespace lq
