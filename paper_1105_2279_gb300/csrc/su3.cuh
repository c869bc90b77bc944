// Device algebra on 3x3 complex matrices (CUDA cores; FMA-form complex
// multiply-accumulate).  Header-only so every kernel inlines it into registers.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

namespace lq {

template <typename R> struct vec2;
template <> struct vec2<float> { typedef float2 type; };
template <> struct vec2<double> { typedef double2 type; };

__device__ __forceinline__ float fmaR(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaR(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename R> struct cx {
  R re, im;
};

template <typename R> __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mkc(a.re + b.re, a.im + b.im); }
template <typename R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mkc(a.re - b.re, a.im - b.im); }
template <typename R> __device__ __forceinline__ cx<R> cconj(cx<R> a) { return mkc(a.re, -a.im); }
template <typename R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mkc(a.re * s, a.im * s); }
// a * b
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mkc(fmaR(a.re, b.re, -a.im * b.im), fmaR(a.re, b.im, a.im * b.re));
}
// c + a * b
template <typename R> __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {
  R re = fmaR(a.re, b.re, c.re);
  R im = fmaR(a.re, b.im, c.im);
  re = fmaR(-a.im, b.im, re);
  im = fmaR(a.im, b.re, im);
  return mkc(re, im);
}
// c + a * conj(b)
template <typename R> __device__ __forceinline__ cx<R> cfma_nc(cx<R> a, cx<R> b, cx<R> c) {
  R re = fmaR(a.re, b.re, c.re);
  R im = fmaR(a.im, b.re, c.im);
  re = fmaR(a.im, b.im, re);
  im = fmaR(-a.re, b.im, im);
  return mkc(re, im);
}
// c + conj(a) * b
template <typename R> __device__ __forceinline__ cx<R> cfma_cn(cx<R> a, cx<R> b, cx<R> c) {
  R re = fmaR(a.re, b.re, c.re);
  R im = fmaR(a.re, b.im, c.im);
  re = fmaR(a.im, b.im, re);
  im = fmaR(-a.im, b.re, im);
  return mkc(re, im);
}

// 3x3 complex matrix, row-major: e[3*row + col].
template <typename R> struct M3 {
  cx<R> e[9];
};

template <typename R> __device__ __forceinline__ void m_zero(M3<R>& m) {
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = mkc<R>(0, 0);
}
template <typename R> __device__ __forceinline__ void m_unit(M3<R>& m) {
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = mkc<R>((i % 4 == 0) ? R(1) : R(0), 0);
}

// C = A B
template <typename R> __device__ __forceinline__ M3<R> mul_nn(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cmul(a.e[3 * i], b.e[k]);
      t = cfma(a.e[3 * i + 1], b.e[3 + k], t);
      c.e[3 * i + k] = cfma(a.e[3 * i + 2], b.e[6 + k], t);
    }
  return c;
}
// C = A B^dag
template <typename R> __device__ __forceinline__ M3<R> mul_nd(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cfma_nc(a.e[3 * i], b.e[3 * k], mkc<R>(0, 0));
      t = cfma_nc(a.e[3 * i + 1], b.e[3 * k + 1], t);
      c.e[3 * i + k] = cfma_nc(a.e[3 * i + 2], b.e[3 * k + 2], t);
    }
  return c;
}
// C = A^dag B
template <typename R> __device__ __forceinline__ M3<R> mul_dn(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cfma_cn(a.e[i], b.e[k], mkc<R>(0, 0));
      t = cfma_cn(a.e[3 + i], b.e[3 + k], t);
      c.e[3 * i + k] = cfma_cn(a.e[6 + i], b.e[6 + k], t);
    }
  return c;
}
// C += A B
template <typename R> __device__ __forceinline__ void mac_nn(M3<R>& c, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cfma(a.e[3 * i], b.e[k], c.e[3 * i + k]);
      t = cfma(a.e[3 * i + 1], b.e[3 + k], t);
      c.e[3 * i + k] = cfma(a.e[3 * i + 2], b.e[6 + k], t);
    }
}
// C += A^dag B
template <typename R> __device__ __forceinline__ void mac_dn(M3<R>& c, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cfma_cn(a.e[i], b.e[k], c.e[3 * i + k]);
      t = cfma_cn(a.e[3 + i], b.e[3 + k], t);
      c.e[3 * i + k] = cfma_cn(a.e[6 + i], b.e[6 + k], t);
    }
}
// C += A B^dag
template <typename R> __device__ __forceinline__ void mac_nd(M3<R>& c, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> t = cfma_nc(a.e[3 * i], b.e[3 * k], c.e[3 * i + k]);
      t = cfma_nc(a.e[3 * i + 1], b.e[3 * k + 1], t);
      c.e[3 * i + k] = cfma_nc(a.e[3 * i + 2], b.e[3 * k + 2], t);
    }
}
template <typename R> __device__ __forceinline__ M3<R> m_adj(const M3<R>& a) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) c.e[3 * i + k] = cconj(a.e[3 * k + i]);
  return c;
}
template <typename R> __device__ __forceinline__ void m_addto(M3<R>& c, const M3<R>& a) {
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = cadd(c.e[i], a.e[i]);
}
template <typename R> __device__ __forceinline__ M3<R> m_add(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = cadd(a.e[i], b.e[i]);
  return c;
}
template <typename R> __device__ __forceinline__ M3<R> m_sub(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = csub(a.e[i], b.e[i]);
  return c;
}
template <typename R> __device__ __forceinline__ M3<R> m_scale(const M3<R>& a, cx<R> s) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = cmul(s, a.e[i]);
  return c;
}
template <typename R> __device__ __forceinline__ M3<R> m_rscale(const M3<R>& a, R s) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 9; ++i) c.e[i] = cscale(a.e[i], s);
  return c;
}
template <typename R> __device__ __forceinline__ cx<R> m_trace(const M3<R>& a) {
  return cadd(cadd(a.e[0], a.e[4]), a.e[8]);
}
// Re tr(A B^dag) = sum_ij Re(A_ij conj(B_ij))
template <typename R> __device__ __forceinline__ R retr_nd(const M3<R>& a, const M3<R>& b) {
  R s = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) s = fmaR(a.e[i].re, b.e[i].re, fmaR(a.e[i].im, b.e[i].im, s));
  return s;
}
// traceless anti-Hermitian part (M - M^dag)/2 - tr(M - M^dag)/6
template <typename R> __device__ __forceinline__ M3<R> m_ta(const M3<R>& m) {
  M3<R> a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> x = m.e[3 * i + k], y = m.e[3 * k + i];
      a.e[3 * i + k] = mkc<R>(R(0.5) * (x.re - y.re), R(0.5) * (x.im + y.im));
    }
  R t = (a.e[0].im + a.e[4].im + a.e[8].im) * R(1.0 / 3.0);
  a.e[0].im -= t;
  a.e[4].im -= t;
  a.e[8].im -= t;
  return a;
}

// ---- structure-of-arrays global memory access ----------------------------
// p points at component 0 of the wanted (dir, site); components are `plane`
// elements apart.
template <typename R>
__device__ __forceinline__ M3<R> ld_m3(const typename vec2<R>::type* __restrict__ p, long long plane) {
  M3<R> m;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    typename vec2<R>::type v = __ldg(p + c * plane);
    m.e[c].re = v.x;
    m.e[c].im = v.y;
  }
  return m;
}
template <typename R>
__device__ __forceinline__ void st_m3(typename vec2<R>::type* __restrict__ p, long long plane, const M3<R>& m) {
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    typename vec2<R>::type v;
    v.x = m.e[c].re;
    v.y = m.e[c].im;
    p[c * plane] = v;
  }
}

}  // namespace lq
