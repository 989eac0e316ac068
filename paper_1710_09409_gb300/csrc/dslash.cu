// The Wilson Dslash hopping term with its spin structure: the operator whose
// port to GPUs the paper names as its next step (Sec. 6, Summary and Outlook),
// beyond the site-local expression engine.
//
//   out(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                   + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
//
// psi and out are spinor fields, stored as colour-vector fields with four
// objects per site (object s = spin component s), U the four links of every
// site.  Euclidean gamma matrices in the chiral basis,
//   gamma_mu = [[0, s_mu], [s_mu^dagger, 0]] in 2x2 spin blocks,
//   s_x = [[0, i], [i, 0]], s_y = [[0, -1], [1, 0]], s_z = [[i, 0], [0, -i]],
//   s_t = 1, so gamma_5 = diag(1, 1, -1, -1).
// (1 + sg gamma_mu) has rank 2: with psi = (u; l) in upper and lower spin
// pairs, (1 + sg gamma_mu) psi = (h; sg s_mu^dagger h) with the half spinor
// h = u + sg s_mu l.  The colour matrix acts on each spin component, so each
// of the 8 terms multiplies only the two components of h by the link (2
// matrix-vector products instead of 4) and rebuilds the lower pair from the
// product.  Every s_mu has one entry per row, a phase in {1, i, -1, -i}, so
// the projection and the rebuild are sums with swapped and negated parts.
//
// Algorithmic traffic per site (FP64, every input read once): the 4 links
// (576 B), the spinor (192 B) and the output (192 B), 960 B; 1320 flops
// (per term: 12 for the projection, 2 x 66 for the products, 24 to
// accumulate; the first term's accumulation is a copy).
#include <cuda_runtime.h>

#include "dev_stencil.cuh"
#include "internal.h"

namespace su3s {

// acc (+)= P * x for a complex x given as (re, im) values, P = i^code.
template <class M, bool FIRST, int CODE>
__device__ __forceinline__ void add_phased(typename M::A& are, typename M::A& aim,
                                           const typename M::R& xr, const typename M::R& xi) {
  if constexpr (CODE == 0) {
    M::template add<FIRST, 1>(are, xr);
    M::template add<FIRST, 1>(aim, xi);
  } else if constexpr (CODE == 1) {  // i (xr + i xi) = -xi + i xr
    M::template add<FIRST, -1>(are, xi);
    M::template add<FIRST, 1>(aim, xr);
  } else if constexpr (CODE == 2) {
    M::template add<FIRST, -1>(are, xr);
    M::template add<FIRST, -1>(aim, xi);
  } else {  // -i (xr + i xi) = xi - i xr
    M::template add<FIRST, 1>(are, xi);
    M::template add<FIRST, -1>(aim, xr);
  }
}

// acc += P * b for an accumulated complex b (two accumulators), P = i^code.
template <class M, int CODE>
__device__ __forceinline__ void combine_phased(typename M::A& are, typename M::A& aim,
                                               const typename M::A& br, const typename M::A& bi) {
  if constexpr (CODE == 0) {
    M::template combine<1>(are, br);
    M::template combine<1>(aim, bi);
  } else if constexpr (CODE == 1) {
    M::template combine<-1>(are, bi);
    M::template combine<1>(aim, br);
  } else if constexpr (CODE == 2) {
    M::template combine<-1>(are, br);
    M::template combine<-1>(aim, bi);
  } else {
    M::template combine<1>(are, bi);
    M::template combine<-1>(aim, br);
  }
}

// h = u + P l for one spin component pair, P = i^ph (ph uniform across the
// warp: one of four compiled forms).
template <class M>
__device__ __forceinline__ void half_spinor(typename M::R* h, const typename M::R* u,
                                            const typename M::R* l, int ph) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    typename M::A re, im;
    M::template add<true, 1>(re, u[2 * c]);
    M::template add<true, 1>(im, u[2 * c + 1]);
    switch (ph) {
      case 0: add_phased<M, false, 0>(re, im, l[2 * c], l[2 * c + 1]); break;
      case 1: add_phased<M, false, 1>(re, im, l[2 * c], l[2 * c + 1]); break;
      case 2: add_phased<M, false, 2>(re, im, l[2 * c], l[2 * c + 1]); break;
      default: add_phased<M, false, 3>(re, im, l[2 * c], l[2 * c + 1]); break;
    }
    h[2 * c] = M::finish(re);
    h[2 * c + 1] = M::finish(im);
  }
}

// out += P chi for a colour vector of accumulators, P = i^ph (uniform).
template <class M>
__device__ __forceinline__ void add_rebuilt(typename M::A* out, const typename M::A* chi, int ph) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    switch (ph) {
      case 0: combine_phased<M, 0>(out[2 * c], out[2 * c + 1], chi[2 * c], chi[2 * c + 1]); break;
      case 1: combine_phased<M, 1>(out[2 * c], out[2 * c + 1], chi[2 * c], chi[2 * c + 1]); break;
      case 2: combine_phased<M, 2>(out[2 * c], out[2 * c + 1], chi[2 * c], chi[2 * c + 1]); break;
      default: combine_phased<M, 3>(out[2 * c], out[2 * c + 1], chi[2 * c], chi[2 * c + 1]); break;
    }
  }
}

template <class M>
__device__ __noinline__ void dslash_site_f64(const FieldDesc& dst, const FieldDesc& U,
                                             const FieldDesc& psi, const LatGeo& g, int64_t s);

// The eight terms at site s, then the store (or, for a site whose inputs are
// outside the FP64-accurate arithmetics' range, native FP64 instead).  The
// terms run in a rolled loop: unrolled, the eight bodies (~10,000 instructions
// per site in the pair arithmetic) overflowed the instruction cache and
// instruction fetch was the leading stall.  Direction and sense are uniform
// across the warp, so the phase and column choices are uniform branches; the
// backward link's adjoint is taken in its load.
template <class M>
__device__ __forceinline__ void dslash_site(const FieldDesc& dst, const FieldDesc& U,
                                            const FieldDesc& psi, const LatGeo& g, int64_t s) {
  typename M::A out[4][6];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int r = 0; r < 6; ++r) out[k][r] = M::zero();
  uint32_t gm = 0;
#pragma unroll 1
  for (int t = 0; t < 8; ++t) {
    const int mu = t >> 1;
    const bool bwd = (t & 1) != 0;          // sense: SG = +1 backward, -1 forward
    const int64_t n = shift_site_rt(g, s, mu, bwd ? -1 : 1);
    // s_mu: row k has its entry in column k ^ sw with phase code ph_k
    const bool sw = mu < 2;
    const int ph0 = mu == 0 ? 1 : mu == 1 ? 2 : mu == 2 ? 1 : 0;
    const int ph1 = mu == 0 ? 1 : mu == 1 ? 0 : mu == 2 ? 3 : 0;
    const int sg = bwd ? 0 : 2;             // phase code of SG
    typename M::R h[2][6];
    {
      typename M::R sp[4][6];
#pragma unroll
      for (int k = 0; k < 4; ++k) load_nc<M, 6>(psi, n, k, sp[k], gm);
      if (sw) {
        half_spinor<M>(h[0], sp[0], sp[3], (ph0 + sg) & 3);
        half_spinor<M>(h[1], sp[1], sp[2], (ph1 + sg) & 3);
      } else {
        half_spinor<M>(h[0], sp[0], sp[2], (ph0 + sg) & 3);
        half_spinor<M>(h[1], sp[1], sp[3], (ph1 + sg) & 3);
      }
    }
    if constexpr (M::kScaled) {
      // fixed point: the half spinor's components share one exponent
      typename M::A a[12];
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < 6; ++r) a[6 * k + r] = M::to_acc(h[k][r]);
      M::template finish_obj<12>(&h[0][0], a);
    }
    typename M::R u[18];
    load_link<M>(U, bwd ? n : s, mu, bwd, u, gm);
    // upper spin k += U h_k; lower spin (k ^ sw) += SG conj(P_k) U h_k
    const int q0 = (((4 - ph0) & 3) + sg) & 3, q1 = (((4 - ph1) & 3) + sg) & 3;
    {
      typename M::A chi[6];
      mv_acc<M, true, 1, false>(chi, u, h[0]);
      add_rebuilt<M>(out[0], chi, 0);
      if (sw) add_rebuilt<M>(out[3], chi, q0);
      else add_rebuilt<M>(out[2], chi, q0);
    }
    {
      typename M::A chi[6];
      mv_acc<M, true, 1, false>(chi, u, h[1]);
      add_rebuilt<M>(out[1], chi, 0);
      if (sw) add_rebuilt<M>(out[2], chi, q1);
      else add_rebuilt<M>(out[3], chi, q1);
    }
  }
  if constexpr (M::kGuard) {
    if (gm >= guard_hi(2)) {
      dslash_site_f64<MathF64>(dst, U, psi, g, s);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const typename M::A(*o)[6] = reinterpret_cast<const typename M::A(*)[6]>(out[k]);
    store_obj<KV, P_F64, M, 1, 6>(dst, s, k, o);
  }
}

template <class M>
__device__ __noinline__ void dslash_site_f64(const FieldDesc& dst, const FieldDesc& U,
                                             const FieldDesc& psi, const LatGeo& g, int64_t s) {
  dslash_site<M>(dst, U, psi, g, s);
}

// One thread per site, a grid of one wave (the neighbours of the sites in
// flight stay in the L2 cache).
template <class M>
__global__ void __launch_bounds__(128) k_dslash(FieldDesc dst, FieldDesc U, FieldDesc psi, LatGeo g) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.V;
       s += (int64_t)gridDim.x * blockDim.x)
    dslash_site<M>(dst, U, psi, g, s);
}

template <class M>
static cudaError_t launch_dslash(const su3s_field* dest, const su3s_field* U, const su3s_field* psi,
                                 cudaStream_t st) {
  const LatGeo g = lat_geo(psi);
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash<M>, 128, 0);
  if (e != cudaSuccess) return e;
  int64_t nb = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();   // one wave
  const int64_t need = (g.V + 127) / 128;
  const dim3 grid((unsigned)(nb < need ? nb : need));
  k_dslash<M><<<grid, 128, 0, st>>>(dest->desc, U->desc, psi->desc, g);
  return cudaGetLastError();
}

}  // namespace su3s

using namespace su3s;

SU3S_EXPORT int su3s_dslash(su3s_field* dest, const su3s_field* U, const su3s_field* psi, int math,
                            void* stream) {
  if (!dest || !U || !psi) return fail(SU3S_EINVAL, "null argument");
  if (U->kind != SU3S_MATRIX || U->nmu != 4)
    return fail(SU3S_ETYPE, "the links must be a matrix field with 4 links per site");
  if (psi->kind != SU3S_VECTOR || psi->nmu != 4 || dest->kind != SU3S_VECTOR || dest->nmu != 4)
    return fail(SU3S_ETYPE, "spinor fields are colour-vector fields with 4 spin components per site");
  if (U->prec != SU3S_F64 || psi->prec != SU3S_F64 || dest->prec != SU3S_F64)
    return fail(SU3S_EUNSUPPORTED, "the Wilson hopping term needs FP64 storage");
  for (int d = 0; d < 4; ++d)
    if (U->L[d] != psi->L[d] || dest->L[d] != psi->L[d])
      return fail(SU3S_ESHAPE, "fields live on different lattices");
  if (overlap(dest, psi) || overlap(dest, U)) return fail(SU3S_EINVAL, "destination overlaps an input");
  if (!valid_math(math)) return fail(SU3S_EINVAL, "bad arithmetic %d", math);
  const int m = resolve_math(SU3S_F64, math);
  cudaStream_t st = (cudaStream_t)stream;
  if (psi->V == 0) return SU3S_OK;
  cudaError_t ce = m == MATH_F64  ? launch_dslash<MathF64>(dest, U, psi, st)
                   : m == MATH_FX ? launch_dslash<MathFX>(dest, U, psi, st)
                                  : launch_dslash<MathDF>(dest, U, psi, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "Wilson hopping-term kernel launch");
  return SU3S_OK;
}
