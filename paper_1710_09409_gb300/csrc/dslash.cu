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

#include <type_traits>

#include "dev_stencil.cuh"
#include "internal.h"

namespace su3s {

// Multiplication by a phase P = i^ph, ph uniform across the warp, without
// branches: P (xr + i xi) = (sr a, si b) with (a, b) = (xr, xi) or (xi, xr)
// (odd ph), sr = -1 for ph = 1, 2 and si = -1 for ph = 2, 3.  Negation is exact
// in every arithmetic, so the result is the phase times the value exactly.
struct Phase {
  bool swap, neg_re, neg_im;
  __device__ __forceinline__ explicit Phase(int ph)
      : swap((ph & 1) != 0), neg_re(ph == 1 || ph == 2), neg_im(ph >= 2) {}
};

template <class M>
__device__ __forceinline__ typename M::A neg_acc(const typename M::A& a) {
  if constexpr (std::is_same<typename M::A, DAcc>::value) return DAcc{-a.S, -a.lo};
  else if constexpr (std::is_same<typename M::A, FAcc>::value) return FAcc{-a.hh, -a.cr, a.e};
  else return -a;
}

// h = u + P l for one spin component pair (colour vectors of reals).
template <class M>
__device__ __forceinline__ void half_spinor(typename M::R* h, const typename M::R* u,
                                            const typename M::R* l, Phase P) {
  if constexpr (M::kPaired) {
    // the pair arithmetic: real and imaginary parts in packed lanes, each lane
    // repeating MathDF::add's operations (the copy, then TwoSum of the
    // leading parts with the tail gathered)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const df a = P.swap ? l[2 * c + 1] : l[2 * c];
      const df b = P.swap ? l[2 * c] : l[2 * c + 1];
      const float2 S = make_float2(u[2 * c].h, u[2 * c + 1].h);
      const float2 lo = make_float2(u[2 * c].l, u[2 * c + 1].l);
      const float2 xh = make_float2(P.neg_re ? -a.h : a.h, P.neg_im ? -b.h : b.h);
      const float2 xl = make_float2(P.neg_re ? -a.l : a.l, P.neg_im ? -b.l : b.l);
      const float2 s = f2_add(S, xh);
      const float2 nbp = f2_sub(S, s);          // -bp
      const float2 ap = f2_add(s, nbp);         // s - bp
      const float2 db = f2_add(xh, nbp);        // xh - bp
      const float2 da = f2_sub(S, ap);
      float2 t = f2_add(da, db);
      t = f2_add(t, xl);
      const float2 lo2 = f2_add(lo, t);
      h[2 * c] = df_norm(s.x, lo2.x);
      h[2 * c + 1] = df_norm(s.y, lo2.y);
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const typename M::R a = P.swap ? l[2 * c + 1] : l[2 * c];
    const typename M::R b = P.swap ? l[2 * c] : l[2 * c + 1];
    typename M::A re, im;
    M::template add<true, 1>(re, u[2 * c]);
    M::template add<true, 1>(im, u[2 * c + 1]);
    M::template add<false, 1>(re, P.neg_re ? M::neg(a) : a);
    M::template add<false, 1>(im, P.neg_im ? M::neg(b) : b);
    h[2 * c] = M::finish(re);
    h[2 * c + 1] = M::finish(im);
  }
}

// out += P chi for a colour vector of accumulators.
template <class M>
__device__ __forceinline__ void add_rebuilt(typename M::A* out, const typename M::A* chi, Phase P) {
  if constexpr (M::kPaired) {
    // real and imaginary parts combined in packed lanes (MathDF::combine per lane)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const DAcc a = P.swap ? chi[2 * c + 1] : chi[2 * c];
      const DAcc b = P.swap ? chi[2 * c] : chi[2 * c + 1];
      DAcc2 o = dacc2_get(out[2 * c], out[2 * c + 1]);
      const DAcc2 x{make_float2(P.neg_re ? -a.S : a.S, P.neg_im ? -b.S : b.S),
                    make_float2(P.neg_re ? -a.lo : a.lo, P.neg_im ? -b.lo : b.lo)};
      df2_combine<1>(o, x);
      dacc2_put(out[2 * c], out[2 * c + 1], o);
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const typename M::A a = P.swap ? chi[2 * c + 1] : chi[2 * c];
    const typename M::A b = P.swap ? chi[2 * c] : chi[2 * c + 1];
    M::template combine<1>(out[2 * c], P.neg_re ? neg_acc<M>(a) : a);
    M::template combine<1>(out[2 * c + 1], P.neg_im ? neg_acc<M>(b) : b);
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
        half_spinor<M>(h[0], sp[0], sp[3], Phase((ph0 + sg) & 3));
        half_spinor<M>(h[1], sp[1], sp[2], Phase((ph1 + sg) & 3));
      } else {
        half_spinor<M>(h[0], sp[0], sp[2], Phase((ph0 + sg) & 3));
        half_spinor<M>(h[1], sp[1], sp[3], Phase((ph1 + sg) & 3));
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
    const Phase q0((((4 - ph0) & 3) + sg) & 3), q1((((4 - ph1) & 3) + sg) & 3), one(0);
    {
      typename M::A chi[6];
      mv_acc<M, true, 1, false>(chi, u, h[0]);
      add_rebuilt<M>(out[0], chi, one);
      if (sw) add_rebuilt<M>(out[3], chi, q0);
      else add_rebuilt<M>(out[2], chi, q0);
    }
    {
      typename M::A chi[6];
      mv_acc<M, true, 1, false>(chi, u, h[1]);
      add_rebuilt<M>(out[1], chi, one);
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

// ------------------------------------------------ staged (asynchronous) loads
// Each thread stages the operands of its next term (the neighbour spinor's 12
// complex components and the link's 9) in its own slots of shared memory with
// asynchronous copies (cp.async) while it computes the current term, so the
// loads' latency is hidden behind a term's arithmetic without holding the
// next operands in registers.  Slots are [element][thread], 16 bytes each.
constexpr int kDslashElems = 21;

// Issue the copies of term t (direction t >> 1, backward if t is odd) of site s.
__device__ __forceinline__ void stage_term(uint4* slot, int nt, const FieldDesc& U,
                                           const FieldDesc& psi, const LatGeo& g, int64_t s, int t) {
  const int mu = t >> 1;
  const bool bwd = (t & 1) != 0;
  const int64_t n = shift_site_rt(g, s, mu, bwd ? -1 : 1);
  const uint4* pp = reinterpret_cast<const uint4*>(psi.ptr);
  const uint4* pu = reinterpret_cast<const uint4*>(U.ptr);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t b = elem_base(psi, n, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) cp_async16(slot + (3 * k + c) * nt, pp + b + c * psi.s_c);
  }
  const int64_t bu = elem_base(U, bwd ? n : s, mu);
#pragma unroll
  for (int e = 0; e < 9; ++e) cp_async16(slot + (12 + e) * nt, pu + bu + e * U.s_c);
  cp_async_commit();
}

template <class M, int W>
__device__ __forceinline__ void read_staged(const uint4* slot, int nt, int first, typename M::R* out,
                                            uint32_t& gm) {
#pragma unroll
  for (int c = 0; c < W / 2; ++c) {
    const uint4 v = slot[(first + c) * nt];
    if constexpr (M::kGuard) gm = guard_max(gm, v.y, v.w);
    split_complex<M>(v, out[2 * c], out[2 * c + 1]);
  }
  M::template normalize_obj<W>(out);
}

// The link of the term from its slots, its adjoint for the backward term
// (element (i, j) read from (j, i), imaginary part negated).
template <class M>
__device__ __forceinline__ void read_staged_link(const uint4* slot, int nt, bool dag,
                                                 typename M::R* out, uint32_t& gm) {
  if (dag) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const uint4 v = slot[(12 + 3 * j + i) * nt];
        if constexpr (M::kGuard) gm = guard_max(gm, v.y, v.w);
        split_complex<M>(make_uint4(v.x, v.y, v.z, v.w ^ 0x80000000u), out[2 * (3 * i + j)],
                         out[2 * (3 * i + j) + 1]);
      }
    M::template normalize_obj<18>(out);
  } else {
    read_staged<M, 18>(slot, nt, 12, out, gm);
  }
}

// The Wilson term at the thread's sites s, s + stride, ...: each term's
// operands were staged during the previous term (the first site's first term
// before the loop), and the next term's copies are issued as soon as this
// term's slots have been read into registers.
template <class M>
__device__ __forceinline__ void dslash_staged(const FieldDesc& dst, const FieldDesc& U,
                                              const FieldDesc& psi, const LatGeo& g, int64_t s,
                                              int64_t stride, uint4* slot, int nt) {
  if (s < g.V) stage_term(slot, nt, U, psi, g, s, 0);
  while (s < g.V) {
    typename M::A out[4][6];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int r = 0; r < 6; ++r) out[k][r] = M::zero();
    uint32_t gm = 0;
#pragma unroll 1
    for (int t = 0; t < 8; ++t) {
      const int mu = t >> 1;
      const bool bwd = (t & 1) != 0;
      const bool sw = mu < 2;
      const int ph0 = mu == 0 ? 1 : mu == 1 ? 2 : mu == 2 ? 1 : 0;
      const int ph1 = mu == 0 ? 1 : mu == 1 ? 0 : mu == 2 ? 3 : 0;
      const int sg = bwd ? 0 : 2;
      cp_async_wait_all();
      typename M::R h[2][6];
      {
        typename M::R sp[4][6];
#pragma unroll
        for (int k = 0; k < 4; ++k) read_staged<M, 6>(slot, nt, 3 * k, sp[k], gm);
        if (sw) {
          half_spinor<M>(h[0], sp[0], sp[3], Phase((ph0 + sg) & 3));
          half_spinor<M>(h[1], sp[1], sp[2], Phase((ph1 + sg) & 3));
        } else {
          half_spinor<M>(h[0], sp[0], sp[2], Phase((ph0 + sg) & 3));
          half_spinor<M>(h[1], sp[1], sp[3], Phase((ph1 + sg) & 3));
        }
      }
      if constexpr (M::kScaled) {
        typename M::A a[12];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int r = 0; r < 6; ++r) a[6 * k + r] = M::to_acc(h[k][r]);
        M::template finish_obj<12>(&h[0][0], a);
      }
      typename M::R u[18];
      read_staged_link<M>(slot, nt, bwd, u, gm);
      // this term's slots are in registers: stage the next term
      if (t < 7) stage_term(slot, nt, U, psi, g, s, t + 1);
      else if (s + stride < g.V) stage_term(slot, nt, U, psi, g, s + stride, 0);
      const Phase q0((((4 - ph0) & 3) + sg) & 3), q1((((4 - ph1) & 3) + sg) & 3), one(0);
      {
        typename M::A chi[6];
        mv_acc<M, true, 1, false>(chi, u, h[0]);
        add_rebuilt<M>(out[0], chi, one);
        if (sw) add_rebuilt<M>(out[3], chi, q0);
        else add_rebuilt<M>(out[2], chi, q0);
      }
      {
        typename M::A chi[6];
        mv_acc<M, true, 1, false>(chi, u, h[1]);
        add_rebuilt<M>(out[1], chi, one);
        if (sw) add_rebuilt<M>(out[2], chi, q1);
        else add_rebuilt<M>(out[3], chi, q1);
      }
    }
    if (M::kGuard && gm >= guard_hi(2)) {
      dslash_site_f64<MathF64>(dst, U, psi, g, s);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const typename M::A(*o)[6] = reinterpret_cast<const typename M::A(*)[6]>(out[k]);
        store_obj<KV, P_F64, M, 1, 6>(dst, s, k, o);
      }
    }
    s += stride;
  }
  cp_async_wait_all();
}

// One thread per site, a grid of one wave (the neighbours of the sites in
// flight stay in the L2 cache), each thread with 21 staging slots.
template <class M>
__global__ void __launch_bounds__(128) k_dslash(FieldDesc dst, FieldDesc U, FieldDesc psi, LatGeo g) {
  extern __shared__ __align__(16) uint4 d_slots[];
  dslash_staged<M>(dst, U, psi, g, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                   (int64_t)gridDim.x * blockDim.x, d_slots + threadIdx.x, (int)blockDim.x);
}

template <class M>
static cudaError_t launch_dslash(const su3s_field* dest, const su3s_field* U, const su3s_field* psi,
                                 cudaStream_t st) {
  const LatGeo g = lat_geo(psi);
  const size_t smem = (size_t)kDslashElems * 16 * 128;
  cudaError_t e = cudaFuncSetAttribute(k_dslash<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  int per_sm = 1;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dslash<M>, 128, smem);
  if (e != cudaSuccess) return e;
  int64_t nb = (int64_t)(per_sm > 0 ? per_sm : 1) * sm_count();   // one wave
  const int64_t need = (g.V + 127) / 128;
  const dim3 grid((unsigned)(nb < need ? nb : need));
  k_dslash<M><<<grid, 128, smem, st>>>(dest->desc, U->desc, psi->desc, g);
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
                                  : launch_dslash<MathDFUnpacked>(dest, U, psi, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "Wilson hopping-term kernel launch");
  return SU3S_OK;
}
