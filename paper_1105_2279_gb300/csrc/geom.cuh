// Lattice geometry shared by every kernel (and by the JIT-compiled expression
// kernels, so this header compiles under NVRTC too): extents, lexicographic
// strides, and periodic neighbours by index arithmetic (no site tables).
#pragma once

namespace lq {

// Geometry parameters passed to kernels by value.
struct GeomArgs {
  int L[4];
  int stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
  int V;
};

__device__ __forceinline__ void site_coords(const GeomArgs& g, int s, int c[4]) {
  int r = s;
  c[0] = r % g.L[0];
  r /= g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}
// c[mu] for a run-time mu without indexing a local array
__device__ __forceinline__ int coord_of(const int c[4], int mu) {
  return mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
}
// site of x + nu, where x has coordinate c_nu along nu
__device__ __forceinline__ int nb_fwd(const GeomArgs& g, int s, int c_nu, int nu) {
  return (c_nu + 1 < g.L[nu]) ? s + g.stride[nu] : s - (g.L[nu] - 1) * g.stride[nu];
}
__device__ __forceinline__ int nb_bwd(const GeomArgs& g, int s, int c_nu, int nu) {
  return (c_nu > 0) ? s - g.stride[nu] : s + (g.L[nu] - 1) * g.stride[nu];
}
// The same for a direction known only at run time: extent and stride picked
// by selects, so the geometry is never indexed (and copied to local memory).
__device__ __forceinline__ int nb_fwd_rt(const GeomArgs& g, int s, int c_nu, int nu) {
  const int L = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
  const int st = nu == 0 ? g.stride[0] : (nu == 1 ? g.stride[1] : (nu == 2 ? g.stride[2] : g.stride[3]));
  return (c_nu + 1 < L) ? s + st : s - (L - 1) * st;
}
__device__ __forceinline__ int nb_bwd_rt(const GeomArgs& g, int s, int c_nu, int nu) {
  const int L = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
  const int st = nu == 0 ? g.stride[0] : (nu == 1 ? g.stride[1] : (nu == 2 ? g.stride[2] : g.stride[3]));
  return (c_nu > 0) ? s - st : s + (L - 1) * st;
}

}  // namespace lq
