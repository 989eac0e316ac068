// Nearest-neighbour operations: the Cshift and the colour part of the Dslash
// hopping term, which the paper names as the next step beyond its site-local
// expression engine (Sec. 6, Summary and Outlook: porting Grid's Dslash
// operator, whose Cshift operations lie outside the expression templates).
//
//   su3s_cshift  dst(x) = src(x + shift e_dim), periodic in every direction:
//                a gather of whole site objects in their storage format.
//   su3s_hop     out(x) = sum_mu U_mu(x) v(x+mu) + U_mu(x-mu)^dagger v(x-mu)
//                for a colour-vector or colour-matrix field v and the four
//                links U of every site, FP64 storage, in the arithmetic of
//                the site-local kernels.
//
// Sites are s = x + Lx (y + Ly (z + Lz t)); one thread per site.  Neighbour
// objects are read through the read-only data cache: every object is read
// by up to eight neighbouring sites, so L1 and L2 supply most of the reuse.
#include <cuda_runtime.h>

#include "dev_stencil.cuh"
#include "internal.h"

namespace su3s {

// ------------------------------------------------------------- Cshift
// One thread per (site, object element); EB bytes per stored element.
template <int EB>
struct Raw;
template <>
struct Raw<16> {
  using T = uint4;
};
template <>
struct Raw<8> {
  using T = uint2;
};
template <>
struct Raw<4> {
  using T = uint32_t;
};

// One thread per site of one element (blockIdx.y = link * ncomp + component);
// consecutive threads take consecutive sites, so reads and writes coalesce
// except where the shift wraps around.
// The shifted direction is passed as its stride and extent (no per-thread
// indexing of the geometry).
template <int EB>
__global__ void __launch_bounds__(256) k_cshift(FieldDesc dst, FieldDesc src, int64_t V,
                                                uint32_t stride, uint32_t extent, int ncomp,
                                                int shift) {
  using T = typename Raw<EB>::T;
  const int q = blockIdx.y;
  const int mu = q / ncomp, c = q - mu * ncomp;
  const int64_t qo_d = (int64_t)mu * dst.s_mu + (int64_t)c * dst.s_c;
  const int64_t qo_s = (int64_t)mu * src.s_mu + (int64_t)c * src.s_c;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t co = (int32_t)(((uint32_t)s / stride) % extent);
    int32_t c2 = co + shift;   // shift in [0, extent)
    c2 = c2 >= (int32_t)extent ? c2 - (int32_t)extent : c2;
    const int64_t n = s + (int64_t)(c2 - co) * stride;
    const T v = __ldg(reinterpret_cast<const T*>(src.ptr) + elem_base(src, n, 0) + qo_s);
    reinterpret_cast<T*>(dst.ptr)[elem_base(dst, s, 0) + qo_d] = v;
  }
}

// ---------------------------------------------------------- hopping term
// The hopping term at site s in the arithmetic M.  Every term's operands are
// range-checked (see dev_math.cuh); a site out of range is computed again in
// native FP64 before its store (the destination overlaps no input).
template <int KIND>
__device__ __noinline__ void hop_site_f64(const FieldDesc& dst, const FieldDesc& U,
                                          const FieldDesc& v, const LatGeo& g, int64_t s);

template <class M, int KIND>
__device__ __forceinline__ void hop_site(const FieldDesc& dst, const FieldDesc& U, const FieldDesc& v,
                                         const LatGeo& g, int64_t s) {
  constexpr int W = KIND == KM ? 18 : 6;
  typename M::A acc[W];
  uint32_t gm = 0;
  if constexpr (KIND == KM) {
#pragma unroll
    for (int r = 0; r < W; ++r) acc[r] = M::zero();
#pragma unroll 1
    for (int t = 0; t < 8; ++t) {
      // t = 2 mu: forward U_mu(x) v(x + mu); t = 2 mu + 1: backward
      // U_mu(x - mu)^dagger v(x - mu)
      const int mu = t >> 1;
      const bool bwd = (t & 1) != 0;
      const int64_t n = shift_site_rt(g, s, mu, bwd ? -1 : 1);
      typename M::R u[18], x[W];
      load_link<M>(U, bwd ? n : s, mu, bwd, u, gm);
      load_nc<M, W>(v, n, 0, x, gm);
      mm_combine<M, 1, false, false>(acc, u, x);
    }
  } else {
    {
      typename M::R u[18], x[W];
      load_nc<M, 18>(U, s, 0, u, gm);
      load_nc<M, W>(v, shift_site_rt(g, s, 0, 1), 0, x, gm);
      mv_acc<M, true, 1, false>(acc, u, x);
    }
#pragma unroll 1
    for (int t = 1; t < 8; ++t) {
      const int mu = t >> 1;
      typename M::R u[18], x[W];
      if ((t & 1) == 0) {
        load_nc<M, 18>(U, s, mu, u, gm);
        load_nc<M, W>(v, shift_site_rt(g, s, mu, 1), 0, x, gm);
        mv_combine<M, 1, false>(acc, u, x);
      } else {
        const int64_t bw = shift_site_rt(g, s, mu, -1);
        load_nc<M, 18>(U, bw, mu, u, gm);
        load_nc<M, W>(v, bw, 0, x, gm);
        mv_combine<M, 1, true>(acc, u, x);
      }
    }
  }
  if constexpr (M::kGuard) {
    if (gm >= guard_hi(2)) {
      hop_site_f64<KIND>(dst, U, v, g, s);
      return;
    }
  }
  typename M::A out[1][W];
#pragma unroll
  for (int r = 0; r < W; ++r) out[0][r] = acc[r];
  store_obj<KIND, P_F64, M, 1, W>(dst, s, 0, out);
}

template <int KIND>
__device__ __noinline__ void hop_site_f64(const FieldDesc& dst, const FieldDesc& U,
                                          const FieldDesc& v, const LatGeo& g, int64_t s) {
  hop_site<MathF64, KIND>(dst, U, v, g, s);
}

// One thread per site; the grid is one wave, so the sites in flight (and the
// backward links and neighbours they share) fit the L2 cache, and the loop over
// the 8 terms is rolled.  Colour matrices: the terms run through a single
// product routine (the backward link's adjoint is taken in its load), which
// keeps the matrix-product code small enough for the instruction cache (+29%
// at 48^4 over separate forward and backward routines).  Colour vectors: the
// matrix-vector code is small, and separate forward and backward routines,
// with the first term opening the accumulators, are faster (+13%).
template <class M, int KIND>
__global__ void __launch_bounds__(128) k_hop(FieldDesc dst, FieldDesc U, FieldDesc v, LatGeo g) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.V;
       s += (int64_t)gridDim.x * blockDim.x)
    hop_site<M, KIND>(dst, U, v, g, s);
}

template <class K>
static dim3 grid_for(K kernel, int threads, int64_t work) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  int64_t nb = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count() * 4;
  const int64_t need = (work + threads - 1) / threads;
  if (nb > need) nb = need;
  return dim3((unsigned)(nb < 1 ? 1 : nb));
}

template <class M, int KIND>
static cudaError_t launch_hop(const su3s_field* dest, const su3s_field* U, const su3s_field* v,
                              cudaStream_t st) {
  const LatGeo g = lat_geo(v);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hop<M, KIND>, 128, 0);
  int64_t nb = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();   // one wave
  const int64_t need = (g.V + 127) / 128;
  const dim3 grid((unsigned)(nb < need ? nb : need));
  k_hop<M, KIND><<<grid, 128, 0, st>>>(dest->desc, U->desc, v->desc, g);
  return cudaGetLastError();
}

}  // namespace su3s

using namespace su3s;

SU3S_EXPORT int su3s_cshift(su3s_field* dest, const su3s_field* src, int dim, int shift,
                            void* stream) {
  if (!dest || !src) return fail(SU3S_EINVAL, "null argument");
  if (dim < 0 || dim > 3) return fail(SU3S_EINVAL, "direction %d is not 0..3", dim);
  int rc = check_same_shape(dest, src, true);
  if (rc) return rc;
  if (dest->kind != src->kind) return fail(SU3S_ETYPE, "fields of different kinds");
  if (overlap(dest, src)) return fail(SU3S_EINVAL, "destination overlaps the source");
  const int L = src->L[dim];
  const int sh = ((shift % L) + L) % L;   // into [0, L)
  const LatGeo g = lat_geo(src);
  const int nelem = src->nmu * src->ncomp;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t ce = cudaSuccess;
  if (g.V == 0) return SU3S_OK;
  const auto grid = [&](dim3 gx) { return dim3(gx.x, (unsigned)nelem, 1); };
  switch (src->elem_bytes) {
    case 16:
      k_cshift<16><<<grid(grid_for(k_cshift<16>, 256, g.V)), 256, 0, st>>>(dest->desc, src->desc, g.V,
                                                                           (uint32_t)g.stride[dim], (uint32_t)g.L[dim], src->ncomp, sh);
      break;
    case 8:
      k_cshift<8><<<grid(grid_for(k_cshift<8>, 256, g.V)), 256, 0, st>>>(dest->desc, src->desc, g.V,
                                                                         (uint32_t)g.stride[dim], (uint32_t)g.L[dim], src->ncomp, sh);
      break;
    default:
      k_cshift<4><<<grid(grid_for(k_cshift<4>, 256, g.V)), 256, 0, st>>>(dest->desc, src->desc, g.V,
                                                                         (uint32_t)g.stride[dim], (uint32_t)g.L[dim], src->ncomp, sh);
      break;
  }
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "cshift kernel launch");
  return SU3S_OK;
}

SU3S_EXPORT int su3s_hop(su3s_field* dest, const su3s_field* U, const su3s_field* v, int math,
                         void* stream) {
  if (!dest || !U || !v) return fail(SU3S_EINVAL, "null argument");
  if (U->kind != SU3S_MATRIX || U->nmu != 4)
    return fail(SU3S_ETYPE, "the links must be a matrix field with 4 links per site");
  if (v->kind == SU3S_REAL || v->nmu != 1)
    return fail(SU3S_ETYPE, "the operand must be a matrix or vector field with one object per site");
  if (dest->kind != v->kind || dest->nmu != 1)
    return fail(SU3S_ETYPE, "the destination must have the operand's kind");
  if (U->prec != SU3S_F64 || v->prec != SU3S_F64 || dest->prec != SU3S_F64)
    return fail(SU3S_EUNSUPPORTED, "the hopping term needs FP64 storage");
  for (int d = 0; d < 4; ++d)
    if (U->L[d] != v->L[d] || dest->L[d] != v->L[d])
      return fail(SU3S_ESHAPE, "fields live on different lattices");
  if (overlap(dest, v) || overlap(dest, U)) return fail(SU3S_EINVAL, "destination overlaps an input");
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  const int m = resolve_math(SU3S_F64, math);
  cudaStream_t st = (cudaStream_t)stream;
  if (v->V == 0) return SU3S_OK;
  cudaError_t ce;
  const bool mat = v->kind == SU3S_MATRIX;
  if (m == MATH_F64) ce = mat ? launch_hop<MathF64, KM>(dest, U, v, st) : launch_hop<MathF64, KV>(dest, U, v, st);
  else if (m == MATH_FX) ce = mat ? launch_hop<MathFX, KM>(dest, U, v, st) : launch_hop<MathFX, KV>(dest, U, v, st);
  else ce = mat ? launch_hop<MathDFScalar, KM>(dest, U, v, st) : launch_hop<MathDF, KV>(dest, U, v, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "hopping-term kernel launch");
  return SU3S_OK;
}
