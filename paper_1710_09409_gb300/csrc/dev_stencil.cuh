// Nearest-neighbour addressing and loads shared by the stencil kernels
// (Cshift, the colour hopping term and the Wilson hopping term with spin).
// Sites are s = x + Lx (y + Ly (z + Lz t)); directions 0..3 are x, y, z, t,
// every direction periodic.
#pragma once

#include <cuda_runtime.h>

#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

struct LatGeo {
  int32_t L[4];
  int32_t stride[4];  // 1, Lx, Lx Ly, Lx Ly Lz
  int64_t V;
};

// Site of s + shift e_dim (periodic); shift in (-L, L).  Volumes are below
// 2^31, so the coordinate arithmetic is 32-bit.
__device__ __forceinline__ int64_t shift_site(const LatGeo& g, int64_t s, int dim, int shift) {
  const uint32_t st = (uint32_t)g.stride[dim], L = (uint32_t)g.L[dim];
  const int32_t c = (int32_t)(((uint32_t)s / st) % L);
  int32_t c2 = c + shift;
  c2 = c2 >= (int32_t)L ? c2 - (int32_t)L : (c2 < 0 ? c2 + (int32_t)L : c2);
  return s + (int64_t)(c2 - c) * st;
}

// FP64 object (W reals) of field f at site s, link mu, through the read-only
// cache, in the arithmetic M.
// g is the site's range guard (largest input high word, see dev_math.cuh).
template <class M, int W>
__device__ __forceinline__ void load_nc(const FieldDesc& f, int64_t s, int mu, typename M::R* out,
                                        uint32_t& g) {
  const int64_t b = elem_base(f, s, mu);
  const uint4* p = reinterpret_cast<const uint4*>(f.ptr);
#pragma unroll
  for (int c = 0; c < W / 2; ++c) {
    const uint4 v = __ldg(p + b + c * f.s_c);
    if constexpr (M::kGuard) g = guard_max(g, v.y, v.w);
    split_complex<M>(v, out[2 * c], out[2 * c + 1]);
  }
  M::template normalize_obj<W>(out);
}

// Link U_mu(s) (dag false) or its adjoint U_mu(s)^dagger (dag true), in the
// arithmetic M.  The adjoint is taken in the load: element (i, j) is read from
// component (j, i) and its imaginary part's sign bit is flipped, so one product
// routine serves the forward and the backward terms.
template <class M>
__device__ __forceinline__ void load_link(const FieldDesc& f, int64_t s, int mu, bool dag,
                                          typename M::R* out, uint32_t& g) {
  const int64_t b = elem_base(f, s, mu);
  const uint4* p = reinterpret_cast<const uint4*>(f.ptr);
  const uint32_t sg = dag ? 0x80000000u : 0u;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int c = 3 * i + j;
      const uint4 v = __ldg(p + b + (dag ? 3 * j + i : c) * f.s_c);
      if constexpr (M::kGuard) g = guard_max(g, v.y, v.w);
      split_complex<M>(make_uint4(v.x, v.y, v.z, v.w ^ sg), out[2 * c], out[2 * c + 1]);
    }
  M::template normalize_obj<18>(out);
}

// Site of s + shift e_mu for a runtime direction (the geometry is selected,
// not indexed, so it stays in registers).
__device__ __forceinline__ int64_t shift_site_rt(const LatGeo& g, int64_t s, int mu, int shift) {
  const uint32_t st = (uint32_t)(mu == 0 ? g.stride[0] : mu == 1 ? g.stride[1] : mu == 2 ? g.stride[2] : g.stride[3]);
  const uint32_t L = (uint32_t)(mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3]);
  const int32_t c = (int32_t)(((uint32_t)s / st) % L);
  int32_t c2 = c + shift;
  c2 = c2 >= (int32_t)L ? c2 - (int32_t)L : (c2 < 0 ? c2 + (int32_t)L : c2);
  return s + (int64_t)(c2 - c) * st;
}

// One thread per site; the grid is one wave, so the sites in flight (and the
// backward links and neighbours they share) fit the L2 cache, and the loop over
// the 8 terms is rolled.  Colour matrices: the terms run through a single
// product routine (the backward link's adjoint is taken in its load), which
// keeps the matrix-product code small enough for the instruction cache (+29%
// at 48^4 over separate forward and backward routines).  Colour vectors: the
// matrix-vector code is small, and separate forward and backward routines,
// with the first term opening the accumulators, are faster (+13%).
// Asynchronous 16-byte copies global -> shared (cp.async), used to stage the
// next term's operands of a stencil while the current term is computed.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

inline LatGeo lat_geo(const su3s_field* f) {
  LatGeo g;
  for (int d = 0; d < 4; ++d) g.L[d] = f->L[d];
  g.stride[0] = 1;
  g.stride[1] = f->L[0];
  g.stride[2] = f->L[0] * f->L[1];
  g.stride[3] = f->L[0] * f->L[1] * f->L[2];
  g.V = f->V;
  return g;
}

inline bool overlap(const su3s_field* a, const su3s_field* b) {
  const char* pa = (const char*)a->ptr;
  const char* pb = (const char*)b->ptr;
  return pa < pb + b->bytes && pb < pa + a->bytes;
}

}  // namespace su3s
