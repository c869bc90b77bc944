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

}  // namespace lq
