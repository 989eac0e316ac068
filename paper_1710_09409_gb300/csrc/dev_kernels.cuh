// Streaming kernels over all sites of a lattice: one pass reads every leaf
// object of a site, evaluates the compiled tree in registers and writes the
// destination object (Sec. 3, Listing 1: _odata[ss] = eval(ss, expr) for
// every ss), and the matching reverse-mode kernel.
//
// Thread mapping follows the vector layout of Sec. 5: consecutive threads of a
// warp take consecutive sites, so every component load of a warp is one
// contiguous 512-byte (FP64) segment; the second grid dimension runs over
// the links mu of Lorentz-indexed fields (the 2-d block of Sec. 5 with the
// "vectors" axis mapped to the grid).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <type_traits>

#include "dev_expr.cuh"
#include "dev_field.cuh"
#include "dev_tma.cuh"
#include "kparams.h"

namespace su3s {

template <int PREC>
struct IsC12 {
  static constexpr bool value = (PREC == P_F64_C12 || PREC == P_F32_C12);
};

// Rebuild row 2 of an SU(3) matrix from rows 0,1: r2_c = conj(r0_j r1_k - r0_k r1_j),
// (c, j, k) cyclic.
template <class M>
__device__ __forceinline__ void rebuild_row2(typename M::R* m) {
  if constexpr (M::kPaired) {
    // the pair arithmetic: the real and imaginary parts of each rebuilt element
    // advance together in packed lanes, each lane repeating the scalar terms
    // below in their order (re: +ajr bkr, -aji bki, -akr bjr, +aki bji; im:
    // -ajr bki, -aji bkr, +akr bji, +aki bjr)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int j = (c + 1) % 3, k = (c + 2) % 3;
      const df ajr = m[2 * j], aji = m[2 * j + 1], akr = m[2 * k], aki = m[2 * k + 1];
      const df bjr = m[6 + 2 * j], bji = m[6 + 2 * j + 1];
      const df bkr = m[6 + 2 * k], bki = m[6 + 2 * k + 1];
      auto pr = [](df x0, bool n0, df x1, bool n1) {
        return df2{make_float2(n0 ? -x0.h : x0.h, n1 ? -x1.h : x1.h),
                   make_float2(n0 ? -x0.l : x0.l, n1 ? -x1.l : x1.l)};
      };
      DAcc2 a;
      df2_first(a, pr(ajr, false, ajr, true), pr(bkr, false, bki, false));
      df2_fma(a, pr(aji, true, aji, true), pr(bki, false, bkr, false));
      df2_fma(a, pr(akr, true, akr, false), pr(bjr, false, bji, false));
      df2_fma(a, pr(aki, false, aki, false), pr(bji, false, bjr, false));
      m[12 + 2 * c] = df_norm(a.S.x, a.lo.x);
      m[12 + 2 * c + 1] = df_norm(a.S.y, a.lo.y);
    }
    return;
  }
  // fixed point: row 2 comes out at the scale of a product; the 18 reals are
  // renormalised together to one shared exponent
  typename M::A a[M::kScaled ? 18 : 1];
  if constexpr (M::kScaled) {
#pragma unroll
    for (int r = 0; r < 12; ++r) a[r] = M::to_acc(m[r]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int j = (c + 1) % 3, k = (c + 2) % 3;
    const typename M::R &ajr = m[2 * j], &aji = m[2 * j + 1];          // r0_j
    const typename M::R &akr = m[2 * k], &aki = m[2 * k + 1];          // r0_k
    const typename M::R &bjr = m[6 + 2 * j], &bji = m[6 + 2 * j + 1];  // r1_j
    const typename M::R &bkr = m[6 + 2 * k], &bki = m[6 + 2 * k + 1];  // r1_k
    typename M::A re, im;
    M::template fma<true, 1>(re, ajr, bkr);
    M::template fma<false, -1>(re, aji, bki);
    M::template fma<false, -1>(re, akr, bjr);
    M::template fma<false, 1>(re, aki, bji);
    // conjugate: imaginary part negated
    M::template fma<true, -1>(im, ajr, bki);
    M::template fma<false, -1>(im, aji, bkr);
    M::template fma<false, 1>(im, akr, bji);
    M::template fma<false, 1>(im, aki, bjr);
    if constexpr (M::kScaled) {
      a[12 + 2 * c] = re;
      a[12 + 2 * c + 1] = im;
    } else {
      m[12 + 2 * c] = M::finish(re);
      m[12 + 2 * c + 1] = M::finish(im);
    }
  }
  if constexpr (M::kScaled) M::template finish_obj<18>(m, a);
}

// Load leaf slot I (kind K) of VPS consecutive sites starting at site s.
template <int K, int PREC, class M, int VPS, class C>
__device__ __forceinline__ void load_obj(const FieldDesc& f, int64_t s, int mu, C* ctx, int slot) {
  const int64_t b = elem_base(f, s, mu);
  if constexpr (K == KR) {
    static_assert(VPS == 1, "real fields are FP64");
    if constexpr (M::kGuard) {
      const uint2 v = ld8((const char*)f.ptr + b * 8);
      ctx[0].gmax = guard_max(ctx[0].gmax, v.y, v.y);
      ctx[0].leaf[slot][0] = M::from_bits(v.x, v.y);
    } else {
      ctx[0].leaf[slot][0] = StoreReal::template load<M>(f.ptr, b);
    }
    M::template normalize_obj<1>(ctx[0].leaf[slot]);
  } else {
    using St = typename BaseStore<PREC>::type;
    constexpr int NC = (K == KV) ? 3 : (IsC12<PREC>::value ? 6 : 9);
    uint32_t gm[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      typename M::R re[VPS], im[VPS];
      if constexpr (M::kGuard) {
        // FP64 storage, one site: the raw words also feed the range guard
        static_assert(VPS == 1, "guarded arithmetics read FP64 storage");
        const uint4 v = ld16((const char*)f.ptr + (b + c * f.s_c) * 16);
        gm[c] = guard_max(0u, v.y, v.w);
        split_complex<M>(v, re[0], im[0]);
      } else {
        St::template load<M>(f.ptr, b + c * f.s_c, re, im);
      }
#pragma unroll
      for (int v = 0; v < VPS; ++v) {
        ctx[v].leaf[slot][2 * c] = re[v];
        ctx[v].leaf[slot][2 * c + 1] = im[v];
      }
    }
    if constexpr (M::kGuard) ctx[0].gmax = max(ctx[0].gmax, guard_reduce<NC>(gm));
    if constexpr (PREC == P_F64 || PREC == P_F64_C12) {
#pragma unroll
      for (int v = 0; v < VPS; ++v) M::template normalize_obj<2 * NC>(ctx[v].leaf[slot]);
    }
    if constexpr (K == KM && IsC12<PREC>::value) {
#pragma unroll
      for (int v = 0; v < VPS; ++v) rebuild_row2<M>(ctx[v].leaf[slot]);
    }
  }
}

template <class Tree, int I, int PREC, class M, int VPS, class C>
__device__ __forceinline__ void load_leaves(const KParams& p, int64_t s, int mu, C* ctx) {
  if constexpr (I < Tree::nleaf) {
    constexpr int K = LeafKind<Tree, I>::value;
    static_assert(K >= 0, "leaf slots must be numbered densely");
    load_obj<K, PREC, M, VPS>(p.leaf[I], s, mu, ctx, I);
    load_leaves<Tree, I + 1, PREC, M, VPS>(p, s, mu, ctx);
  }
}

// Store accumulators acc[v][W] of VPS sites into field f.
template <int K, int PREC, class M, int VPS, int W>
__device__ __forceinline__ void store_obj(const FieldDesc& f, int64_t s, int mu,
                                          const typename M::A (*acc)[W]) {
  const int64_t b = elem_base(f, s, mu);
  if constexpr (K == KR) {
    StoreReal::template store_acc<M>(f.ptr, b, acc[0][0]);
  } else {
    using St = typename BaseStore<PREC>::type;
    constexpr int NC = (K == KV) ? 3 : (IsC12<PREC>::value ? 6 : 9);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      typename M::A re[VPS], im[VPS];
#pragma unroll
      for (int v = 0; v < VPS; ++v) {
        re[v] = acc[v][2 * c];
        im[v] = acc[v][2 * c + 1];
      }
      St::template store_acc<M>(f.ptr, b + c * f.s_c, re, im);
    }
  }
}

template <int PREC>
struct Vps {
  static constexpr int value = BaseStore<PREC>::type::VPS;
};
template <>
struct Vps<P_F64> {
  static constexpr int value = 1;
};

// ------------------------------------------------------------ forward kernel
// Native FP64 evaluation of one site from its inputs in global memory: the
// range guard's path for sites outside the FP64-accurate arithmetics' range.
// Kept out of line so that it costs the hot loop neither code nor registers.
template <class Tree, int PREC>
__device__ __noinline__ void eval_site_f64(const KParams& p, int64_t s, int mu);

template <class Tree, class M, int PREC>
__device__ __forceinline__ void eval_sites(const KParams& p, int64_t t, int mu) {
  constexpr int VPS = Vps<PREC>::value;
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int W = Width<Tree::kind>::value;
  Ctx<M, NL, NS> ctx[VPS];
#pragma unroll
  for (int v = 0; v < VPS; ++v) {
#pragma unroll
    for (int k = 0; k < (NS > 0 ? NS : 1); ++k)
      ctx[v].sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
    ctx[v].gmax = p.gscal;
  }
  const int64_t s = t * VPS;
  load_leaves<Tree, 0, PREC, M, VPS>(p, s, mu, ctx);
  if constexpr (M::kGuard) {
    if (guard_trips<Tree>(ctx[0].gmax)) {
      eval_site_f64<Tree, PREC>(p, s, mu);
      return;
    }
  }
  typename M::A acc[VPS][W];
#pragma unroll
  for (int v = 0; v < VPS; ++v) {
    if constexpr (Tree::accumulates) {
      acc_into<Tree, M, true, 1>(ctx[v], acc[v]);
    } else {
      typename M::R val[W];
      value<Tree, M>(ctx[v], val);
#pragma unroll
      for (int r = 0; r < W; ++r) acc[v][r] = M::to_acc(val[r]);
    }
  }
  store_obj<Tree::kind, PREC, M, VPS, W>(p.dst, s, mu, acc);
}

// Evaluation context of one site that loads each leaf from global memory
// when the evaluation reads it (plain loads), so that only the operands in use
// are held in registers: the range guard's native FP64 path, which runs inside
// kernels tuned for another arithmetic and should not raise their register
// count.
template <class Tree, class M, int PREC>
struct GlobalCtx {
  static constexpr int NS = Tree::nsc;
  const KParams* p;
  int64_t s;
  int mu;
  typename M::R sc[NS > 0 ? NS : 1];
  template <int I, int W>
  __device__ __forceinline__ void leaf_value(typename M::R* out) const {
    Ctx<M, 1, 0> tmp[1];
    load_obj<LeafKind<Tree, I>::value, PREC, M, 1>(p->leaf[I], s, mu, tmp, 0);
#pragma unroll
    for (int r = 0; r < W; ++r) out[r] = tmp[0].leaf[0][r];
  }
};

template <class Tree, int PREC>
__device__ __noinline__ void eval_site_f64(const KParams& p, int64_t s, int mu) {
  using M = MathF64;
  constexpr int W = Width<Tree::kind>::value;
  GlobalCtx<Tree, M, PREC> ctx{&p, s, mu};
#pragma unroll
  for (int k = 0; k < (Tree::nsc > 0 ? Tree::nsc : 1); ++k) ctx.sc[k] = p.sc[k];
  typename M::A acc[1][W];
  if constexpr (Tree::accumulates) {
    acc_into<Tree, M, true, 1>(ctx, acc[0]);
  } else {
    typename M::R val[W];
    value<Tree, M>(ctx, val);
#pragma unroll
    for (int r = 0; r < W; ++r) acc[0][r] = val[r];
  }
  store_obj<Tree::kind, PREC, M, 1, W>(p.dst, s, mu, acc);
}

// Units of work a thread (plain loads: site vectors) or a warp (staged: 32-site
// tiles) takes: first, first + stride, ... below end.
struct Range {
  int64_t first, end, stride;
};

__device__ __forceinline__ Range thread_range(int64_t end) {
  return Range{(int64_t)blockIdx.x * blockDim.x + threadIdx.x, end,
               (int64_t)gridDim.x * blockDim.x};
}
__device__ __forceinline__ Range warp_range(int64_t end) {
  const int nw = blockDim.x >> 5;
  return Range{(int64_t)blockIdx.x * nw + (threadIdx.x >> 5), end, (int64_t)gridDim.x * nw};
}

template <class Tree, class M, int PREC>
__device__ __forceinline__ void plain_range(const KParams& p, Range r) {
  const int mu = blockIdx.y;
  for (int64_t t = r.first; t < r.end; t += r.stride) eval_sites<Tree, M, PREC>(p, t, mu);
}

template <class Tree, class M, int PREC>
__global__ void __launch_bounds__(256) k_eval(const __grid_constant__ KParams p) {
  plain_range<Tree, M, PREC>(p, thread_range(p.nvec));
}

// ------------------------------------------------------------ reverse kernel
template <class Tree, class M>
struct GradSink {
  const GParams* p;
  int64_t s;
  int mu;
  template <int I, int W>
  __device__ __forceinline__ void put(const typename M::A* a) {
    const FieldDesc& f = p->gleaf[I];
    if (f.ptr == nullptr) return;
    const typename M::A(*acc)[W] = reinterpret_cast<const typename M::A(*)[W]>(a);
    store_obj<LeafKind<Tree, I>::value, P_F64, M, 1, W>(f, s, mu, acc);
  }
};

template <class Tree, int I, class M, class GA, class Sink>
__device__ __forceinline__ void store_repeated(GA& ga, Sink& sink) {
  if constexpr (I < Tree::nleaf) {
    if constexpr (Count<Tree, I>::value > 1) {
      constexpr int W = Width<LeafKind<Tree, I>::value>::value;
      sink.template put<I, W>(ga.g[I]);
    }
    store_repeated<Tree, I + 1, M>(ga, sink);
  }
}

// Native FP64 reverse mode of one site (the range guard's path; out of line).
// It reads the leaves and dL/dZ again from global memory, so the gradient
// fields must not overlap them (su3s_eval_adjoint checks).
template <class Tree>
__device__ __noinline__ void adj_site_f64(const GParams& p, int64_t s, int mu);

template <class Tree, class M>
__device__ __forceinline__ void adj_site(const GParams& p, int64_t s, int mu) {
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  Ctx<M, NL, NS> ctx[1];
#pragma unroll
  for (int k = 0; k < (NS > 0 ? NS : 1); ++k)
    ctx[0].sc[k] = M::scalar(p.k.sc[k], p.k.sch[k], p.k.scl[k]);
  ctx[0].gmax = p.k.gscal;
  load_leaves<Tree, 0, P_F64, M, 1>(p.k, s, mu, ctx);
  // dL/dZ
  Ctx<M, 1, 0> g[1];
  load_obj<Tree::kind, P_F64, M, 1>(p.gout, s, mu, g, 0);
  if constexpr (M::kGuard) {
    if (guard_trips<Tree>(max(ctx[0].gmax, g[0].gmax))) {
      adj_site_f64<Tree>(p, s, mu);
      return;
    }
  }
  GradAcc<M, NL> ga;
#pragma unroll
  for (int i = 0; i < NL; ++i)
#pragma unroll
    for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
  GradSink<Tree, M> sink{&p, s, mu};
  Rev<Tree>::template run<Tree, M>(ctx[0], g[0].leaf[0], ga, sink);
  store_repeated<Tree, 0, M>(ga, sink);
}

template <class Tree>
__device__ __noinline__ void adj_site_f64(const GParams& p, int64_t s, int mu) {
  using M = MathF64;
  constexpr int NL = Tree::nleaf;
  GlobalCtx<Tree, M, P_F64> ctx{&p.k, s, mu};
#pragma unroll
  for (int k = 0; k < (Tree::nsc > 0 ? Tree::nsc : 1); ++k) ctx.sc[k] = p.k.sc[k];
  Ctx<M, 1, 0> g[1];
  load_obj<Tree::kind, P_F64, M, 1>(p.gout, s, mu, g, 0);
  GradAcc<M, NL> ga;
#pragma unroll
  for (int i = 0; i < NL; ++i)
#pragma unroll
    for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
  GradSink<Tree, M> sink{&p, s, mu};
  Rev<Tree>::template run<Tree, M>(ctx, g[0].leaf[0], ga, sink);
  store_repeated<Tree, 0, M>(ga, sink);
}

template <class Tree, class M>
__device__ __forceinline__ void adj_plain_range(const GParams& p, Range rg) {
  const int mu = blockIdx.y;
  for (int64_t s = rg.first; s < rg.end; s += rg.stride) adj_site<Tree, M>(p, s, mu);
}

template <class Tree, class M>
__global__ void __launch_bounds__(256) k_adjoint(const __grid_constant__ GParams p) {
  adj_plain_range<Tree, M>(p, thread_range(p.k.nvec));
}

// ------------------------------------------------- TMA-staged variants
// FP64 storage.  Each warp owns a 32-site tile buffer in shared memory: it
// waits for its tile, reads its sites into registers, immediately asks the
// TMA engine for the next tile, and computes while the copy is in flight.
// One lane issues one 2-D tensor copy per matrix or vector object: the
// field's tensor map has rows of 32 consecutive sites of one component
// (64 doubles; rows of one object are Vpad apart in the SoA layout and the
// site block apart in the site-blocked one), so an object's tile is a box of
// (components x 64 doubles) landing as [component][site] in shared memory.

template <int K, int PREC>
struct StageBytes {
  static constexpr int value =
      K == KR ? 256 : (K == KV ? 3 : (IsC12<PREC>::value ? 6 : 9)) * 512;
};

template <class Tree, int PREC, int I>
struct LeafOff {
  static constexpr int value =
      LeafOff<Tree, PREC, I - 1>::value + StageBytes<LeafKind<Tree, I - 1>::value, PREC>::value;
};
template <class Tree, int PREC>
struct LeafOff<Tree, PREC, 0> {
  static constexpr int value = 0;
};

// bytes of one staged tile: the leaves, plus dL/dZ for reverse mode
template <class Tree, int PREC, bool GRAD>
struct TileBytes {
  static constexpr int value = LeafOff<Tree, PREC, Tree::nleaf>::value +
                               (GRAD ? StageBytes<Tree::kind, PREC>::value : 0);
};

// Shared memory of one warp in the whole-tile variant: the tile, then its
// barrier, padded so every warp's buffer starts on a 128-byte boundary.
__host__ __device__ constexpr int tma_warp_stride(int tile_bytes) {
  return (tile_bytes + 16 + 127) / 128 * 128;
}

// Stage one object (kind K) of the 32-site tile starting at site s0, link mu,
// into dst (one lane): matrix and vector objects are one 2-D tensor copy of
// all their components (rows of the field's tensor map), real objects one
// 256-byte bulk copy.
template <int K, int PREC>
__device__ __forceinline__ void issue_obj(const FieldDesc& f, const CUtensorMap* tm, int64_t s0,
                                          int mu, unsigned char* dst, uint64_t* bar) {
  if constexpr (K == KR) {
    const int64_t e = elem_base(f, s0, mu);
    tma_load_1d(dst, (const char*)f.ptr + e * 8, 256, bar);
  } else {
    const int x = 2 * (int)(s0 & (int64_t)f.mask);  // column in doubles: 16-byte aligned
    const int y = (int)((s0 >> f.logB) * f.row_blk + (int64_t)mu * f.row_mu);
    tma_load_2d(dst, tm, x, y, bar);
  }
}

template <class Tree, int I, int PREC>
__device__ __forceinline__ void issue_leaves(const KParams& p, int64_t s0, int mu,
                                             unsigned char* buf, uint64_t* bar) {
  if constexpr (I < Tree::nleaf) {
    issue_obj<LeafKind<Tree, I>::value, PREC>(p.leaf[I], &p.tm[I], s0, mu,
                                              buf + LeafOff<Tree, PREC, I>::value, bar);
    issue_leaves<Tree, I + 1, PREC>(p, s0, mu, buf, bar);
  }
}

// Whole tile: one lane arms the barrier with the tile's bytes and issues one
// copy per object (dL/dZ last in reverse mode).
template <class Tree, int PREC, bool GRAD>
__device__ __forceinline__ void issue_tile(int lane, const KParams& p, const FieldDesc* gout,
                                           const CUtensorMap* tm_gout, int64_t s0, int mu,
                                           unsigned char* buf, uint64_t* bar) {
  constexpr int NL = Tree::nleaf;
  if (lane == 0) {
    mbar_arrive_expect_tx(bar, TileBytes<Tree, PREC, GRAD>::value);
    issue_leaves<Tree, 0, PREC>(p, s0, mu, buf, bar);
    if constexpr (GRAD)
      issue_obj<Tree::kind, PREC>(*gout, tm_gout, s0, mu, buf + LeafOff<Tree, PREC, NL>::value, bar);
  }
  __syncwarp();
}

// Read this lane's site of a staged object into ctx.leaf[slot].
template <int K, int PREC, class M, class C>
__device__ __forceinline__ void read_obj(const unsigned char* src, int lane, C& ctx, int slot) {
  if constexpr (K == KR) {
    const uint2 v = reinterpret_cast<const uint2*>(src)[lane];
    if constexpr (M::kGuard) ctx.gmax = guard_max(ctx.gmax, v.y, v.y);
    ctx.leaf[slot][0] = M::from_bits(v.x, v.y);
    M::template normalize_obj<1>(ctx.leaf[slot]);
  } else {
    constexpr int NC = StageBytes<K, PREC>::value / 512;
    uint32_t gm[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const uint4 v = reinterpret_cast<const uint4*>(src + c * 512)[lane];
      if constexpr (M::kGuard) gm[c] = guard_max(0u, v.y, v.w);
      split_complex<M>(v, ctx.leaf[slot][2 * c], ctx.leaf[slot][2 * c + 1]);
    }
    if constexpr (M::kGuard) ctx.gmax = max(ctx.gmax, guard_reduce<NC>(gm));
    M::template normalize_obj<2 * NC>(ctx.leaf[slot]);
    if constexpr (K == KM && IsC12<PREC>::value) rebuild_row2<M>(ctx.leaf[slot]);
  }
}

template <class Tree, int I, int PREC, class M, class C>
__device__ __forceinline__ void read_leaves(const unsigned char* buf, int lane, C& ctx) {
  if constexpr (I < Tree::nleaf) {
    read_obj<LeafKind<Tree, I>::value, PREC, M>(buf + LeafOff<Tree, PREC, I>::value, lane, ctx, I);
    read_leaves<Tree, I + 1, PREC, M>(buf, lane, ctx);
  }
}

// Sums and differences of two products over disjoint leaves (a*b + c*d): the
// whole-tile kernels read the first product's leaves, evaluate it, and only
// then read the second's (the tile's buffer is refilled once the last leaf is
// read), so the two products' operands are never live together.  The
// evaluation is acc_node's for such a sum: the first product into the
// accumulators, the second combined (mul_combine).
template <class X, class Y, int I>
constexpr bool disjoint_leaves() {
  if constexpr (I >= kMaxLeaves) return true;
  else return (Count<X, I>::value == 0 || Count<Y, I>::value == 0) && disjoint_leaves<X, Y, I + 1>();
}
template <class T>
struct TwoProducts {
  static constexpr bool value = false;
};
template <class X, class Y, int SG>
struct TwoProductsOf {
  static constexpr bool value =
      IsMulNode<X>::value && IsMulNode<Y>::value && disjoint_leaves<X, Y, 0>();
  using P0 = X;
  using P1 = Y;
  static constexpr int S1 = SG;
};
template <class X, class Y>
struct TwoProducts<Add<X, Y>> : TwoProductsOf<X, Y, 1> {};
template <class X, class Y>
struct TwoProducts<Sub<X, Y>> : TwoProductsOf<X, Y, -1> {};

// Sums and differences of two 3x3 products whose leaves overlap
// (adj(a)*b - b*adj(a)): every leaf stays live through both products, so the
// whole-tile kernel evaluates the output one row at a time -- the first
// product's row into three accumulators, the second's row combined into them,
// the row converted and stored -- and holds three outputs' accumulators
// instead of the eighteen of both products.  Each output's operations are
// acc_node's and mul_combine's in the same order: the values are unchanged.
// Pair arithmetic with packed (re, im) lanes, full FP64 matrices.
template <class T>
struct MatLeafOperand {
  static constexpr bool value = false;
};
template <int J>
struct MatLeafOperand<LM<J>> {
  static constexpr bool value = true, adj = false;
  static constexpr int slot = J;
};
template <int J>
struct MatLeafOperand<Adj<LM<J>>> {
  static constexpr bool value = true, adj = true;
  static constexpr int slot = J;
};
template <class T>
struct MatLeafProduct {
  static constexpr bool value = false;
};
template <class X, class Y>
struct MatLeafProduct<Mul<X, Y>> {
  using LX = MatLeafOperand<X>;
  using LY = MatLeafOperand<Y>;
  static constexpr bool value = LX::value && LY::value;
};
template <class T>
struct RowProducts {
  static constexpr bool value = false;
};
template <class X, class Y, int SG>
struct RowProductsOf {
  static constexpr bool value =
      MatLeafProduct<X>::value && MatLeafProduct<Y>::value && !disjoint_leaves<X, Y, 0>();
  using P0 = MatLeafProduct<X>;
  using P1 = MatLeafProduct<Y>;
  static constexpr int S1 = SG;
};
template <class X, class Y>
struct RowProducts<Add<X, Y>> : RowProductsOf<X, Y, 1> {};
template <class X, class Y>
struct RowProducts<Sub<X, Y>> : RowProductsOf<X, Y, -1> {};

template <class Tree, class M, int PREC>
struct RowProductsOk {
  static constexpr bool value = RowProducts<Tree>::value && M::kPaired && PREC == P_F64;
};

// Evaluate and store site s, row by row (RowProductsOk holds).
template <class Tree, class M, class C>
__device__ __forceinline__ void row_products_store(const FieldDesc& f, const C& ctx, int64_t s,
                                                   int mu) {
  using RP = RowProducts<Tree>;
  using X0 = typename RP::P0::LX;
  using Y0 = typename RP::P0::LY;
  using X1 = typename RP::P1::LX;
  using Y1 = typename RP::P1::LY;
  const int64_t b = elem_base(f, s, mu);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    DAcc2 P[3], Q[3];
    mm_pairs_row2<X0::adj, Y0::adj, X1::adj, Y1::adj>(P, Q, ctx.leaf[X0::slot], ctx.leaf[Y0::slot],
                                                      ctx.leaf[X1::slot], ctx.leaf[Y1::slot], i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      df2_combine<RP::S1>(P[k], Q[k]);
      typename M::A re, im;
      dacc2_put(re, im, P[k]);
      Store<P_F64>::template store_acc<M>(f.ptr, b + (3 * i + k) * f.s_c, &re, &im);
    }
  }
}

// Read the staged leaves of subtree Sub (this lane's site) into ctx.
template <class Tree, class Sub, int I, int PREC, class M, class C>
__device__ __forceinline__ void read_leaves_of(const unsigned char* buf, int lane, C& ctx) {
  if constexpr (I < Tree::nleaf) {
    if constexpr (Count<Sub, I>::value > 0)
      read_obj<LeafKind<Tree, I>::value, PREC, M>(buf + LeafOff<Tree, PREC, I>::value, lane, ctx, I);
    read_leaves_of<Tree, Sub, I + 1, PREC, M>(buf, lane, ctx);
  }
}

template <class Tree, class M, int PREC>
__device__ __forceinline__ void tma_range(const KParams& p, Range rg, unsigned char* smem) {
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int W = Width<Tree::kind>::value;
  constexpr int TB = TileBytes<Tree, PREC, false>::value;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = smem + warp * tma_warp_stride(TB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + TB);
  const int mu = blockIdx.y;
  const int64_t ntiles = rg.end;
  const int64_t wstride = rg.stride;
  int64_t t = rg.first;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  if (t < ntiles) issue_tile<Tree, PREC, false>(lane, p, nullptr, nullptr, t << 5, mu, buf, bar);
  Ctx<M, NL, NS> ctx;
#pragma unroll
  for (int k = 0; k < (NS > 0 ? NS : 1); ++k) ctx.sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
  uint32_t phase = 0;
  while (t < ntiles) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, phase));
    if (!ok) {
      if (lane == 0) report_timeout(p.err, bar, phase);
      break;
    }
    phase ^= 1;
    ctx.gmax = p.gscal;
    const int64_t tn = t + wstride;
    if constexpr (RowProductsOk<Tree, M, PREC>::value) {
      read_leaves<Tree, 0, PREC, M>(buf, lane, ctx);
      fence_proxy_async_smem();
      __syncwarp();
      if (tn < ntiles) issue_tile<Tree, PREC, false>(lane, p, nullptr, nullptr, tn << 5, mu, buf, bar);
      if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(ctx.gmax)))
        eval_site_f64<Tree, PREC>(p, (t << 5) + lane, mu);
      else
        row_products_store<Tree, M>(p.dst, ctx, (t << 5) + lane, mu);
      t = tn;
      continue;
    }
    if constexpr (TwoProducts<Tree>::value) {
      using TP = TwoProducts<Tree>;
      typename M::A acc[1][W];
      read_leaves_of<Tree, typename TP::P0, 0, PREC, M>(buf, lane, ctx);
      acc_into<typename TP::P0, M, true, 1>(ctx, acc[0]);
      read_leaves_of<Tree, typename TP::P1, 0, PREC, M>(buf, lane, ctx);
      fence_proxy_async_smem();
      __syncwarp();
      if (tn < ntiles) issue_tile<Tree, PREC, false>(lane, p, nullptr, nullptr, tn << 5, mu, buf, bar);
      // the range is known once every leaf is read; nothing is stored yet
      if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(ctx.gmax))) {
        eval_site_f64<Tree, PREC>(p, (t << 5) + lane, mu);
      } else {
        mul_combine<M, TP::S1>(ctx, acc[0], (typename TP::P1*)nullptr);
        store_obj<Tree::kind, PREC, M, 1, W>(p.dst, (t << 5) + lane, mu, acc);
      }
      t = tn;
      continue;
    }
    read_leaves<Tree, 0, PREC, M>(buf, lane, ctx);
    fence_proxy_async_smem();
    __syncwarp();
    if (tn < ntiles) issue_tile<Tree, PREC, false>(lane, p, nullptr, nullptr, tn << 5, mu, buf, bar);
    // a tile with a site out of range runs all its sites in native FP64: the
    // decision is warp-uniform, so the hot path has no divergent branch
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(ctx.gmax))) {
      eval_site_f64<Tree, PREC>(p, (t << 5) + lane, mu);
    } else {
      typename M::A acc[1][W];
      if constexpr (Tree::accumulates) {
        acc_into<Tree, M, true, 1>(ctx, acc[0]);
      } else {
        typename M::R val[W];
        value<Tree, M>(ctx, val);
#pragma unroll
        for (int r = 0; r < W; ++r) acc[0][r] = M::to_acc(val[r]);
      }
      store_obj<Tree::kind, PREC, M, 1, W>(p.dst, (t << 5) + lane, mu, acc);
    }
    t = tn;
  }
}

// Minimum blocks per SM the whole-tile kernel declares, which steers the
// registers ptxas gives it: row-by-row products fit 128 registers (two blocks
// of 256 threads); the other full-matrix trees in the pair arithmetic are given
// the registers of one block (more independent work per warp: a*b+c*d 234
// instead of 186 registers at the same 8 warps per SM, and measured faster);
// two-row matrices and the other arithmetics state no minimum (two-row a*b: 107
// registers and many warps, 10% faster than with one block's 148).
template <class Tree, class M, int PREC>
struct TmaMinBlocks {
  static constexpr int value = RowProductsOk<Tree, M, PREC>::value        ? 2
                               : (PREC == P_F64 && M::kPaired) ? 1
                                                                : 0;
};

template <class Tree, class M, int PREC>
__global__ void __launch_bounds__(256, TmaMinBlocks<Tree, M, PREC>::value)
    k_eval_tma(const __grid_constant__ KParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.err)) return;
  tma_range<Tree, M, PREC>(p, warp_range(p.nvec >> 5), smem);
}

template <class Tree, class M>
__device__ __forceinline__ void adj_tma_range(const GParams& p, Range rg, unsigned char* smem) {
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int TB = TileBytes<Tree, P_F64, true>::value;
  constexpr int GOFF = LeafOff<Tree, P_F64, NL>::value;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = smem + warp * tma_warp_stride(TB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + TB);
  const int mu = blockIdx.y;
  const int64_t ntiles = rg.end;
  const int64_t wstride = rg.stride;
  int64_t t = rg.first;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  if (t < ntiles) issue_tile<Tree, P_F64, true>(lane, p.k, &p.gout, &p.tm_gout, t << 5, mu, buf, bar);
  Ctx<M, NL, NS> ctx;
#pragma unroll
  for (int k = 0; k < (NS > 0 ? NS : 1); ++k)
    ctx.sc[k] = M::scalar(p.k.sc[k], p.k.sch[k], p.k.scl[k]);
  uint32_t phase = 0;
  while (t < ntiles) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, phase));
    if (!ok) {
      if (lane == 0) report_timeout(p.k.err, bar, phase);
      break;
    }
    phase ^= 1;
    ctx.gmax = p.k.gscal;
    read_leaves<Tree, 0, P_F64, M>(buf, lane, ctx);
    Ctx<M, 1, 0> g;
    read_obj<Tree::kind, P_F64, M>(buf + GOFF, lane, g, 0);
    fence_proxy_async_smem();
    __syncwarp();
    const int64_t tn = t + wstride;
    if (tn < ntiles) issue_tile<Tree, P_F64, true>(lane, p.k, &p.gout, &p.tm_gout, tn << 5, mu, buf, bar);
    {
      GradAcc<M, NL> ga;
#pragma unroll
      for (int i = 0; i < NL; ++i)
#pragma unroll
        for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
      GradSink<Tree, M> sink{&p, (t << 5) + lane, mu};
      Rev<Tree>::template run<Tree, M>(ctx, g.leaf[0], ga, sink);
      store_repeated<Tree, 0, M>(ga, sink);
    }
    // the gradients overlap no input, so a tile with a site out of range is
    // rewritten in native FP64 after the pass (no branch ahead of it)
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(max(ctx.gmax, g.gmax))))
      adj_site_f64<Tree>(p, (t << 5) + lane, mu);
    t = tn;
  }
}

template <class Tree, class M>
__global__ void __launch_bounds__(256) k_adjoint_tma(const __grid_constant__ GParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.k.err)) return;
  adj_tma_range<Tree, M>(p, warp_range(p.k.nvec >> 5), smem);
}

// ------------------------------------------- lazily staged (per-leaf) variant
// Each leaf has its own buffer and mbarrier per warp.  A leaf is read from
// shared memory when the evaluator first needs it; a leaf used once has its
// buffer refilled with the next tile right after that read, a leaf used more
// than once after the tile is computed.  Register pressure follows the
// evaluation order (as with plain loads) while copies overlap compute.
// Times leaf slot I is read from its buffer per tile: once per occurrence in
// forward evaluation; in reverse mode a product also re-reads the leaves of a
// composite operand when it back-propagates into it.
template <class T, int I>
struct RevReads {
  static constexpr int value = 0;
};
template <class X, class Y, int I>
struct RevReads<Mul<X, Y>, I> {
  using BX = typename Operand<X>::base;
  using BY = typename Operand<Y>::base;
  static constexpr int value =
      Count<BX, I>::value + Count<BY, I>::value + RevReads<BX, I>::value + RevReads<BY, I>::value;
};
template <class X, class Y, int I>
struct RevReads<Add<X, Y>, I> {
  static constexpr int value = RevReads<X, I>::value + RevReads<Y, I>::value;
};
template <class X, class Y, int I>
struct RevReads<Sub<X, Y>, I> {
  static constexpr int value = RevReads<X, I>::value + RevReads<Y, I>::value;
};
template <int K, class X, int I>
struct RevReads<Scale<K, X>, I> {
  static constexpr int value = RevReads<X, I>::value;
};
template <class X, int I>
struct RevReads<Adj<X>, I> {
  static constexpr int value = RevReads<X, I>::value;
};
template <class Tree, int I, bool GRAD>
struct Reads {
  static constexpr int value =
      GRAD ? (Tree::is_leaf ? Count<Tree, I>::value : RevReads<Tree, I>::value) : Count<Tree, I>::value;
};

template <class Tree, int PREC, bool GRAD>
struct LazyLayout {
  static constexpr int NL = Tree::nleaf;
  static constexpr int NB = NL + (GRAD ? 1 : 0);   // barriers
  static constexpr int DATA = TileBytes<Tree, PREC, GRAD>::value;
  static constexpr int BYTES = DATA + 8 * NB;      // + one barrier per buffer
  static constexpr int STRIDE = (BYTES + 127) / 128 * 128;
};

template <class Tree, class M, int PREC, bool GRAD>
struct LazyCtx {
  using L = LazyLayout<Tree, PREC, GRAD>;
  static constexpr int NL = Tree::nleaf;
  static constexpr int NS = Tree::nsc;
  unsigned char* buf;
  uint64_t* bars;
  const KParams* p;
  const FieldDesc* gout;
  const CUtensorMap* tm_gout;
  int64_t next_s0;
  int mu, lane;
  uint32_t parity;
  bool has_next;
  mutable bool dead;
  mutable uint32_t gmax;  // range guard of the current tile's site
  typename M::R sc[NS > 0 ? NS : 1];

  template <int I>
  __device__ __forceinline__ void issue(int64_t s0) const {
    constexpr int K = I < NL ? LeafKind<Tree, I>::value : Tree::kind;
    constexpr int OFF = LeafOff<Tree, PREC, I>::value;
    if (lane == 0) {
      mbar_arrive_expect_tx(&bars[I], StageBytes<K, PREC>::value);
      const FieldDesc& f = I < NL ? p->leaf[I < NL ? I : 0] : *gout;
      const CUtensorMap* tm = I < NL ? &p->tm[I < NL ? I : 0] : tm_gout;
      issue_obj<K, PREC>(f, tm, s0, mu, buf + OFF, &bars[I]);
    }
    __syncwarp();
  }

  // wait for leaf I of the current tile (bounded; a time-out marks the warp dead)
  template <int I>
  __device__ __forceinline__ void wait_leaf() const {
    if (dead) return;
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[I], parity));
    if (!ok) {
      if (lane == 0 && p->err) atomicExch(p->err, kErrTmaTimeout);
      dead = true;
    }
  }

  template <int I, int W>
  __device__ __forceinline__ void leaf_value(typename M::R* out) const {
    constexpr int K = I < NL ? LeafKind<Tree, I>::value : Tree::kind;
    wait_leaf<I>();
    Ctx<M, 1, 0> tmp;
    read_obj<K, PREC, M>(buf + LeafOff<Tree, PREC, I>::value, lane, tmp, 0);
    if constexpr (M::kGuard) gmax = max(gmax, tmp.gmax);
#pragma unroll
    for (int r = 0; r < W; ++r) out[r] = tmp.leaf[0][r];
    if constexpr (I >= NL || Reads<Tree, (I < NL ? I : 0), GRAD>::value == 1) {
      // single use: hand the buffer back for the next tile now
      fence_proxy_async_smem();
      __syncwarp();
      if (has_next && !dead) issue<I>(next_s0);
    }
  }

  // after the tile: refill leaves used more than once
  template <int I>
  __device__ __forceinline__ void refill_repeated() const {
    if constexpr (I < NL) {
      if constexpr (Reads<Tree, I, GRAD>::value != 1) {
        fence_proxy_async_smem();
        __syncwarp();
        if (has_next && !dead) issue<I>(next_s0);
      }
      refill_repeated<I + 1>();
    }
  }

  template <int I>
  __device__ __forceinline__ void issue_all(int64_t s0) const {
    if constexpr (I < L::NB) {
      issue<I>(s0);
      issue_all<I + 1>(s0);
    }
  }

  // after a time-out: let copies in flight land (bounded), once per barrier
  template <int I>
  __device__ __forceinline__ void drain() const {
    if constexpr (I < L::NB) {
      mbar_wait_bounded(&bars[I], parity);
      drain<I + 1>();
    }
  }
};

template <class Tree, class M, int PREC, bool GRAD>
__device__ __forceinline__ void lazy_setup(LazyCtx<Tree, M, PREC, GRAD>& c, unsigned char* smem,
                                           const KParams& p, const FieldDesc* gout,
                                           const CUtensorMap* tm_gout) {
  using L = LazyLayout<Tree, PREC, GRAD>;
  const int warp = threadIdx.x >> 5;
  c.lane = threadIdx.x & 31;
  c.buf = smem + warp * L::STRIDE;
  c.bars = reinterpret_cast<uint64_t*>(c.buf + L::DATA);
  c.p = &p;
  c.gout = gout;
  c.tm_gout = tm_gout;
  c.mu = blockIdx.y;
  c.parity = 0;
  c.dead = false;
  if (c.lane == 0) {
#pragma unroll
    for (int i = 0; i < L::NB; ++i) mbar_init(&c.bars[i], 1);
    fence_barrier_init();
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (Tree::nsc > 0 ? Tree::nsc : 1); ++k)
    c.sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
}

template <class Tree, class M, int PREC>
__device__ __forceinline__ void lazy_range(const KParams& p, Range rg, unsigned char* smem) {
  constexpr int W = Width<Tree::kind>::value;
  LazyCtx<Tree, M, PREC, false> c;
  lazy_setup(c, smem, p, nullptr, nullptr);
  const int64_t ntiles = rg.end;
  const int64_t wstride = rg.stride;
  int64_t t = rg.first;
  if (t < ntiles) c.template issue_all<0>(t << 5);
  while (t < ntiles) {
    const int64_t tn = t + wstride;
    c.has_next = tn < ntiles;
    c.next_s0 = tn << 5;
    c.gmax = p.gscal;
    typename M::A acc[1][W];
    if constexpr (Tree::accumulates) {
      acc_into<Tree, M, true, 1>(c, acc[0]);
    } else {
      typename M::R val[W];
      value<Tree, M>(c, val);
#pragma unroll
      for (int r = 0; r < W; ++r) acc[0][r] = M::to_acc(val[r]);
    }
    c.template refill_repeated<0>();
    if (c.dead) break;
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(c.gmax)))
      eval_site_f64<Tree, PREC>(p, (t << 5) + c.lane, c.mu);
    else store_obj<Tree::kind, PREC, M, 1, W>(p.dst, (t << 5) + c.lane, c.mu, acc);
    c.parity ^= 1;
    t = tn;
  }
  if (c.dead) c.template drain<0>();
}

template <class Tree, class M, int PREC>
__global__ void __launch_bounds__(128, 3) k_eval_lazy(const __grid_constant__ KParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.err)) return;
  lazy_range<Tree, M, PREC>(p, warp_range(p.nvec >> 5), smem);
}

template <class Tree, class M>
__device__ __forceinline__ void adj_lazy_range(const GParams& p, Range rg, unsigned char* smem) {
  constexpr int NL = Tree::nleaf;
  constexpr int W = Width<Tree::kind>::value;
  LazyCtx<Tree, M, P_F64, true> c;
  lazy_setup(c, smem, p.k, &p.gout, &p.tm_gout);
  const int64_t ntiles = rg.end;
  const int64_t wstride = rg.stride;
  int64_t t = rg.first;
  if (t < ntiles) c.template issue_all<0>(t << 5);
  while (t < ntiles) {
    const int64_t tn = t + wstride;
    c.has_next = tn < ntiles;
    c.next_s0 = tn << 5;
    c.gmax = p.k.gscal;
    typename M::R G[W];
    c.template leaf_value<NL, W>(G);   // dL/dZ
    GradAcc<M, NL> ga;
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
    GradSink<Tree, M> sink{&p, (t << 5) + c.lane, c.mu};
    Rev<Tree>::template run<Tree, M>(c, G, ga, sink);
    store_repeated<Tree, 0, M>(ga, sink);
    c.template refill_repeated<0>();
    if (c.dead) break;
    // leaves are read as the reverse pass needs them, so the range is known
    // only now: a site out of range overwrites its gradients in native FP64
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(c.gmax)))
      adj_site_f64<Tree>(p, (t << 5) + c.lane, c.mu);
    c.parity ^= 1;
    t = tn;
  }
  if (c.dead) c.template drain<0>();
}

template <class Tree, class M>
__global__ void __launch_bounds__(128, 3) k_adjoint_lazy(const __grid_constant__ GParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.k.err)) return;
  adj_lazy_range<Tree, M>(p, warp_range(p.k.nvec >> 5), smem);
}

// ------------------------------------------- ring-staged variant
// For trees that read every object (leaf, and dL/dZ in reverse mode) exactly
// once per tile, in an order fixed at compile time: K <= (objects) rotating
// buffers per warp, position j of a tile's read order using buffer j % K.
// Reading position j frees its buffer for that buffer's next position: j + K
// of this tile if there is one, else position j % K of the warp's next tile.
// Each copy then has about K positions' worth of compute to land, while a
// warp holds K object buffers instead of one per object.

// Read order of leaf slots, as lists built at compile time.
struct SlotSeq {
  int s[16];
  int n;
};
__host__ __device__ constexpr SlotSeq seq_empty() { return SlotSeq{{0}, 0}; }
__host__ __device__ constexpr SlotSeq seq_one(int slot) {
  SlotSeq r{{0}, 1};
  r.s[0] = slot;
  return r;
}
__host__ __device__ constexpr SlotSeq seq_cat(SlotSeq a, SlotSeq b) {
  for (int i = 0; i < b.n && a.n < 16; ++i) a.s[a.n++] = b.s[i];
  return a;
}
__host__ __device__ constexpr SlotSeq seq_cat(SlotSeq a, SlotSeq b, SlotSeq c, SlotSeq d) {
  return seq_cat(seq_cat(a, b), seq_cat(c, d));
}

// Forward evaluation reads operands left to right (value, acc_into).
template <class T>
struct FwdSeq {
  __host__ __device__ static constexpr SlotSeq get() { return seq_one(T::slot); }
};
template <class X, class Y>
struct FwdSeq<Mul<X, Y>> {
  __host__ __device__ static constexpr SlotSeq get() {
    return seq_cat(FwdSeq<typename Operand<X>::base>::get(), FwdSeq<typename Operand<Y>::base>::get());
  }
};
template <class X, class Y>
struct FwdSeq<Add<X, Y>> {
  __host__ __device__ static constexpr SlotSeq get() { return seq_cat(FwdSeq<X>::get(), FwdSeq<Y>::get()); }
};
template <class X, class Y>
struct FwdSeq<Sub<X, Y>> {
  __host__ __device__ static constexpr SlotSeq get() { return seq_cat(FwdSeq<X>::get(), FwdSeq<Y>::get()); }
};
template <int K, class X>
struct FwdSeq<Scale<K, X>> {
  __host__ __device__ static constexpr SlotSeq get() { return FwdSeq<X>::get(); }
};
template <class X>
struct FwdSeq<Adj<X>> {
  __host__ __device__ static constexpr SlotSeq get() { return FwdSeq<X>::get(); }
};

// Reverse mode (Rev::run): a product reads Y's value, back-propagates into X,
// reads X's value, back-propagates into Y; leaves read nothing.
template <class T>
struct RevSeq {
  __host__ __device__ static constexpr SlotSeq get() { return seq_empty(); }
};
template <class X, class Y>
struct RevSeq<Mul<X, Y>> {
  using BX = typename Operand<X>::base;
  using BY = typename Operand<Y>::base;
  __host__ __device__ static constexpr SlotSeq get() {
    return seq_cat(FwdSeq<BY>::get(), RevSeq<BX>::get(), FwdSeq<BX>::get(), RevSeq<BY>::get());
  }
};
template <class X, class Y>
struct RevSeq<Add<X, Y>> {
  __host__ __device__ static constexpr SlotSeq get() { return seq_cat(RevSeq<X>::get(), RevSeq<Y>::get()); }
};
template <class X, class Y>
struct RevSeq<Sub<X, Y>> {
  __host__ __device__ static constexpr SlotSeq get() { return seq_cat(RevSeq<X>::get(), RevSeq<Y>::get()); }
};
template <int K, class X>
struct RevSeq<Scale<K, X>> {
  __host__ __device__ static constexpr SlotSeq get() { return RevSeq<X>::get(); }
};
template <class X>
struct RevSeq<Adj<X>> {
  __host__ __device__ static constexpr SlotSeq get() { return RevSeq<X>::get(); }
};

// Objects of a tile in read order; dL/dZ is slot nleaf and comes first.
template <class Tree, bool GRAD>
struct ReadSeq {
  __host__ __device__ static constexpr SlotSeq get() {
    if constexpr (GRAD) return seq_cat(seq_one(Tree::nleaf), RevSeq<Tree>::get());
    else return FwdSeq<Tree>::get();
  }
};

template <class Tree, bool GRAD>
__host__ __device__ constexpr int seq_pos(int slot) {
  constexpr SlotSeq q = ReadSeq<Tree, GRAD>::get();
  for (int i = 0; i < q.n; ++i)
    if (q.s[i] == slot) return i;
  return -1;
}

// Whether every object is read exactly once (the ring's requirement).
template <class Tree, bool GRAD>
__host__ __device__ constexpr bool ring_ok() {
  constexpr SlotSeq q = ReadSeq<Tree, GRAD>::get();
  constexpr int nobj = Tree::nleaf + (GRAD ? 1 : 0);
  bool ok = q.n == nobj && nobj >= 3;
  for (int slot = 0; slot < nobj; ++slot) {
    int c = 0;
    for (int i = 0; i < q.n; ++i) c += q.s[i] == slot;
    ok = ok && c == 1;
  }
  return ok;
}

// Position that buffer j % K serves after position j of a tile (n objects):
// j + K of the same tile, else j % K of the next tile.
__host__ __device__ constexpr int ring_next(int j, int n, int K) { return j + K < n ? j + K : j % K; }

// The schedule, checked at compile time over three tiles: every buffer
// alternates strictly between one copy in flight and one read.
template <class Tree, bool GRAD, int K>
__host__ __device__ constexpr bool ring_schedule_ok() {
  constexpr int n = Tree::nleaf + (GRAD ? 1 : 0);
  int busy[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // copies in flight per buffer
  for (int j = 0; j < K && j < n; ++j) busy[j % K] += 1;
  for (int t = 0; t < 3; ++t)
    for (int j = 0; j < n; ++j) {
      const int b = j % K;
      if (busy[b] != 1) return false;  // the read must find exactly its copy
      busy[b] = 0;
      const int nj = ring_next(j, n, K);
      if (nj % K != b) return false;
      busy[b] += 1;
    }
  return true;
}

template <class Tree, int PREC, bool GRAD>
struct RingLayout {
  static constexpr int NOBJ = Tree::nleaf + (GRAD ? 1 : 0);
  static constexpr int K = NOBJ > 3 ? 3 : NOBJ;                   // buffers per warp
  static constexpr int BUF = StageBytes<KM, PREC>::value;         // largest object
  static constexpr int DATA = K * BUF;
  static constexpr int STRIDE = (DATA + 8 * K + 127) / 128 * 128;
};

template <class Tree, class M, int PREC, bool GRAD>
struct RingCtx {
  using L = RingLayout<Tree, PREC, GRAD>;
  static constexpr int NL = Tree::nleaf;
  static constexpr int NS = Tree::nsc;
  static constexpr SlotSeq kSeq = ReadSeq<Tree, GRAD>::get();
  static_assert(ring_schedule_ok<Tree, GRAD, L::K>(), "ring schedule reuses a busy buffer");
  unsigned char* buf;
  uint64_t* bars;
  const KParams* p;
  const FieldDesc* gout;
  const CUtensorMap* tm_gout;
  int64_t cur_s0, next_s0;
  int mu, lane;
  mutable uint32_t ph;  // barrier parity of each buffer
  bool has_next;
  mutable bool dead;
  mutable uint32_t gmax;  // range guard of the current tile's site
  typename M::R sc[NS > 0 ? NS : 1];

  template <int I>
  __device__ __forceinline__ void issue(int64_t s0, int b) const {
    constexpr int K = I < NL ? LeafKind<Tree, (I < NL ? I : 0)>::value : Tree::kind;
    if (lane == 0) {
      mbar_arrive_expect_tx(&bars[b], StageBytes<K, PREC>::value);
      const FieldDesc& f = I < NL ? p->leaf[I < NL ? I : 0] : *gout;
      const CUtensorMap* tm = I < NL ? &p->tm[I < NL ? I : 0] : tm_gout;
      issue_obj<K, PREC>(f, tm, s0, mu, buf + b * L::BUF, &bars[b]);
    }
    __syncwarp();
  }

  // issue the object at position j of the tile whose first site is s0
  template <int J>
  __device__ __forceinline__ void issue_pos(int64_t s0) const {
    issue<kSeq.s[J]>(s0, J % L::K);
  }

  template <int I, int W>
  __device__ __forceinline__ void leaf_value(typename M::R* out) const {
    constexpr int j = seq_pos<Tree, GRAD>(I);
    static_assert(j >= 0, "object outside the read order");
    constexpr int b = j % L::K;
    constexpr int K = I < NL ? LeafKind<Tree, (I < NL ? I : 0)>::value : Tree::kind;
    if (!dead) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[b], (ph >> b) & 1u));
      if (!ok) {
        if (lane == 0 && p->err) atomicExch(p->err, kErrTmaTimeout);
        dead = true;
      }
    }
    ph ^= 1u << b;
    Ctx<M, 1, 0> tmp;
    read_obj<K, PREC, M>(buf + b * L::BUF, lane, tmp, 0);
    if constexpr (M::kGuard) gmax = max(gmax, tmp.gmax);
#pragma unroll
    for (int r = 0; r < W; ++r) out[r] = tmp.leaf[0][r];
    fence_proxy_async_smem();
    __syncwarp();
    if (dead) return;
    // hand the buffer to its next position (this tile, else the next one)
    constexpr int nj = ring_next(j, L::NOBJ, L::K);
    if constexpr (nj > j) issue_pos<nj>(cur_s0);
    else if (has_next) issue_pos<nj>(next_s0);
  }

  template <int J>
  __device__ __forceinline__ void issue_first(int64_t s0) const {
    if constexpr (J < L::K) {
      issue_pos<J>(s0);
      issue_first<J + 1>(s0);
    }
  }

  // after a time-out: let copies in flight land (bounded), once per buffer
  __device__ __forceinline__ void drain() const {
#pragma unroll
    for (int b = 0; b < L::K; ++b) mbar_wait_bounded(&bars[b], (ph >> b) & 1u);
  }
};

template <class Tree, class M, int PREC, bool GRAD>
__device__ __forceinline__ void ring_setup(RingCtx<Tree, M, PREC, GRAD>& c, unsigned char* smem,
                                           const KParams& p, const FieldDesc* gout,
                                           const CUtensorMap* tm_gout) {
  using L = RingLayout<Tree, PREC, GRAD>;
  const int warp = threadIdx.x >> 5;
  c.lane = threadIdx.x & 31;
  c.buf = smem + warp * L::STRIDE;
  c.bars = reinterpret_cast<uint64_t*>(c.buf + L::DATA);
  c.p = &p;
  c.gout = gout;
  c.tm_gout = tm_gout;
  c.mu = blockIdx.y;
  c.ph = 0;
  c.dead = false;
  if (c.lane == 0) {
#pragma unroll
    for (int i = 0; i < L::K; ++i) mbar_init(&c.bars[i], 1);
    fence_barrier_init();
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < (Tree::nsc > 0 ? Tree::nsc : 1); ++k)
    c.sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
}

template <class Tree, class M, int PREC>
__device__ __forceinline__ void ring_range(const KParams& p, Range rg, unsigned char* smem) {
  constexpr int W = Width<Tree::kind>::value;
  RingCtx<Tree, M, PREC, false> c;
  ring_setup(c, smem, p, nullptr, nullptr);
  const int64_t ntiles = rg.end;
  int64_t t = rg.first;
  if (t < ntiles) c.template issue_first<0>(t << 5);
  while (t < ntiles) {
    const int64_t tn = t + rg.stride;
    c.cur_s0 = t << 5;
    c.has_next = tn < ntiles;
    c.next_s0 = tn << 5;
    c.gmax = p.gscal;
    typename M::A acc[1][W];
    if constexpr (Tree::accumulates) {
      acc_into<Tree, M, true, 1>(c, acc[0]);
    } else {
      typename M::R val[W];
      value<Tree, M>(c, val);
#pragma unroll
      for (int r = 0; r < W; ++r) acc[0][r] = M::to_acc(val[r]);
    }
    if (c.dead) break;
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(c.gmax)))
      eval_site_f64<Tree, PREC>(p, (t << 5) + c.lane, c.mu);
    else store_obj<Tree::kind, PREC, M, 1, W>(p.dst, (t << 5) + c.lane, c.mu, acc);
    t = tn;
  }
  if (c.dead) c.drain();
}

template <class Tree, class M, int PREC>
__global__ void __launch_bounds__(128, 4) k_eval_ring(const __grid_constant__ KParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.err)) return;
  ring_range<Tree, M, PREC>(p, warp_range(p.nvec >> 5), smem);
}

template <class Tree, class M>
__device__ __forceinline__ void adj_ring_range(const GParams& p, Range rg, unsigned char* smem) {
  constexpr int NL = Tree::nleaf;
  constexpr int W = Width<Tree::kind>::value;
  RingCtx<Tree, M, P_F64, true> c;
  ring_setup(c, smem, p.k, &p.gout, &p.tm_gout);
  const int64_t ntiles = rg.end;
  int64_t t = rg.first;
  if (t < ntiles) c.template issue_first<0>(t << 5);
  while (t < ntiles) {
    const int64_t tn = t + rg.stride;
    c.cur_s0 = t << 5;
    c.has_next = tn < ntiles;
    c.next_s0 = tn << 5;
    c.gmax = p.k.gscal;
    typename M::R G[W];
    c.template leaf_value<NL, W>(G);   // dL/dZ
    GradAcc<M, NL> ga;
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
    GradSink<Tree, M> sink{&p, (t << 5) + c.lane, c.mu};
    Rev<Tree>::template run<Tree, M>(c, G, ga, sink);
    store_repeated<Tree, 0, M>(ga, sink);
    if (c.dead) break;
    // as in the per-leaf variant: the range is known after the reverse pass
    if (M::kGuard && __any_sync(0xffffffffu, guard_trips<Tree>(c.gmax)))
      adj_site_f64<Tree>(p, (t << 5) + c.lane, c.mu);
    t = tn;
  }
  if (c.dead) c.drain();
}

template <class Tree, class M>
__global__ void __launch_bounds__(128, 3) k_adjoint_ring(const __grid_constant__ GParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.k.err)) return;
  adj_ring_range<Tree, M>(p, warp_range(p.k.nvec >> 5), smem);
}

// ------------------------------------------------------------ launchers
using LaunchFn = cudaError_t (*)(const void* params, dim3 grid, dim3 block, cudaStream_t st);

template <class Tree, class M, int PREC>
cudaError_t launch_eval(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  k_eval<Tree, M, PREC><<<grid, block, 0, st>>>(*static_cast<const KParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M>
cudaError_t launch_adjoint(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  k_adjoint<Tree, M><<<grid, block, 0, st>>>(*static_cast<const GParams*>(params));
  return cudaGetLastError();
}

// Largest dynamic shared memory a block may opt into on the current device.
inline int smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        n <= 0)
      n = 48 * 1024;
    v = n;
  }
  return v;
}

// Dynamic shared memory of a TMA-staged launch: one tile buffer and one
// barrier per warp.
inline size_t tma_smem(int tile_bytes, dim3 block) {
  return (size_t)(block.x / 32) * tma_warp_stride(tile_bytes);
}

template <class Tree, class M, int PREC>
cudaError_t launch_eval_tma(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int TB = TileBytes<Tree, PREC, false>::value;
  const size_t sm = tma_smem(TB, block);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eval_tma<Tree, M, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * tma_warp_stride(TB));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_eval_tma<Tree, M, PREC><<<grid, block, sm, st>>>(*static_cast<const KParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M>
cudaError_t launch_adjoint_tma(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int TB = TileBytes<Tree, P_F64, true>::value;
  const size_t sm = tma_smem(TB, block);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_tma<Tree, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * tma_warp_stride(TB));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_adjoint_tma<Tree, M><<<grid, block, sm, st>>>(*static_cast<const GParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M, int PREC>
cudaError_t launch_eval_lazy(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = LazyLayout<Tree, PREC, false>::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eval_lazy<Tree, M, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * S);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_eval_lazy<Tree, M, PREC><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const KParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M>
cudaError_t launch_adjoint_lazy(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = LazyLayout<Tree, P_F64, true>::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_lazy<Tree, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * S);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_adjoint_lazy<Tree, M><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const GParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M, int PREC>
cudaError_t launch_eval_ring(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = RingLayout<Tree, PREC, false>::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eval_ring<Tree, M, PREC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * S);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_eval_ring<Tree, M, PREC><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const KParams*>(params));
  return cudaGetLastError();
}

template <class Tree, class M>
cudaError_t launch_adjoint_ring(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = RingLayout<Tree, P_F64, true>::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_ring<Tree, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * S);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_adjoint_ring<Tree, M><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const GParams*>(params));
  return cudaGetLastError();
}

// ------------------------------------------------------------ signatures
// Canonical text of a tree type; the host builds the same text from a runtime
// tree (leaves numbered by first appearance, factors in left-to-right order).
template <class T>
struct Sig;
template <int I>
struct Sig<LM<I>> {
  static std::string str() { return "M" + std::to_string(I); }
};
template <int I>
struct Sig<LV<I>> {
  static std::string str() { return "V" + std::to_string(I); }
};
template <int I>
struct Sig<LR<I>> {
  static std::string str() { return "R" + std::to_string(I); }
};
template <class X, class Y>
struct Sig<Mul<X, Y>> {
  static std::string str() { return "mul(" + Sig<X>::str() + "," + Sig<Y>::str() + ")"; }
};
template <class X, class Y>
struct Sig<Add<X, Y>> {
  static std::string str() { return "add(" + Sig<X>::str() + "," + Sig<Y>::str() + ")"; }
};
template <class X, class Y>
struct Sig<Sub<X, Y>> {
  static std::string str() { return "sub(" + Sig<X>::str() + "," + Sig<Y>::str() + ")"; }
};
template <int K, class X>
struct Sig<Scale<K, X>> {
  static std::string str() { return "scale(s" + std::to_string(K) + "," + Sig<X>::str() + ")"; }
};
template <class X>
struct Sig<Adj<X>> {
  static std::string str() { return "adj(" + Sig<X>::str() + ")"; }
};

// Registry hooks implemented by the library (api.cu).  A TMA-staged variant
// (null for reduced-precision storage) is registered beside the plain one,
// with its tile bytes per warp.
// Default launch of a tree when the caller set none: data movement variant,
// threads per block, blocks per SM (0: as many as fit, or one site per thread
// for plain loads).  The rule restates the fastest candidates of the
// autotuner (su3s_tune, su3s_tune_adjoint) on the GB300 at 48^4, FP64 storage;
// trees without staged kernels (reduced precisions) always use plain loads.
struct DefaultGeo {
  int variant, threads, bps;
};
// A product of two distinct leaves (either may be an adjoint).
template <class T>
struct IsLeafProduct {
  static constexpr bool value = false;
};
template <class T, bool LEAF = T::is_leaf>
struct SlotOf {
  static constexpr int value = -1;
};
template <class T>
struct SlotOf<T, true> {
  static constexpr int value = T::slot;
};
template <class X, class Y>
struct IsLeafProduct<Mul<X, Y>> {
  using BX = typename Operand<X>::base;
  using BY = typename Operand<Y>::base;
  static constexpr bool value =
      BX::is_leaf && BY::is_leaf && SlotOf<BX>::value != SlotOf<BY>::value;
};

}  // namespace su3s

#include "dev_pairs.cuh"

namespace su3s {

template <class Tree, class M, int PREC, bool GRAD>
constexpr DefaultGeo default_geometry() {
  // With one tensor copy per object, whole-tile staging is the fastest data
  // movement for every FP64 tree measured, in both FP64-accurate arithmetics,
  // except the reverse mode of a product of two matrix leaves in the pair
  // arithmetic: two sites per lane.  Forward products of two leaves run best
  // in small blocks, about 8 warps per SM (16 for matrix times vector); the
  // rest with the most that fit.
  if constexpr (M::kScaled) return DefaultGeo{1, 128, 0};
  else if constexpr (GRAD && pair_adjoint_ok<Tree, M>()) return DefaultGeo{4, 256, 0};
  else if constexpr (!GRAD && PREC == P_F64 && IsLeafProduct<Tree>::value)
    return Tree::kind == KV ? DefaultGeo{1, 64, 8} : DefaultGeo{1, 64, 4};
  else return DefaultGeo{1, 256, 0};
}

template <class Tree>
cudaError_t launch_eval_pair(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = PairEvalLayout<Tree>::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eval_pair<Tree>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * S < smem_optin() ? 8 * S : smem_optin());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_eval_pair<Tree><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const KParams*>(params));
  return cudaGetLastError();
}

template <class Tree>
cudaError_t launch_adjoint_pair(const void* params, dim3 grid, dim3 block, cudaStream_t st) {
  constexpr int S = PairAdjLayout::STRIDE;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint_pair<Tree>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * S < smem_optin() ? 8 * S : smem_optin());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_adjoint_pair<Tree><<<grid, block, (block.x / 32) * S, st>>>(*static_cast<const GParams*>(params));
  return cudaGetLastError();
}

// Kernel variants of one tree: 0 plain loads, 1 TMA-staged eagerly (whole
// tile), 2 TMA-staged lazily (per leaf), 3 TMA-staged through a ring of
// buffers (trees that read each object once), 4 TMA-staged two tiles at a
// time with two sites per lane (the pair arithmetic on products of matrix
// leaves).  1-4 exist for FP64 storage.
struct Variants {
  LaunchFn fn[5];
  const void* kernel[5];
  int warp_bytes[5];  // shared memory per warp (0 for plain loads)
  int default_variant;
  int default_threads;  // 0: library default
  int default_bps;
};
void register_eval(const std::string& sig, int prec, int math, const Variants& v, int vps);
void register_adjoint(const std::string& sig, int math, const Variants& v);

template <class Tree, class M, int PREC>
void reg_eval(int math) {
  Variants v{};
  v.fn[0] = &launch_eval<Tree, M, PREC>;
  v.kernel[0] = (const void*)&k_eval<Tree, M, PREC>;
  if constexpr (PREC == P_F64 || PREC == P_F64_C12) {
    v.fn[1] = &launch_eval_tma<Tree, M, PREC>;
    v.kernel[1] = (const void*)&k_eval_tma<Tree, M, PREC>;
    v.warp_bytes[1] = tma_warp_stride(TileBytes<Tree, PREC, false>::value);
    v.fn[2] = &launch_eval_lazy<Tree, M, PREC>;
    v.kernel[2] = (const void*)&k_eval_lazy<Tree, M, PREC>;
    v.warp_bytes[2] = LazyLayout<Tree, PREC, false>::STRIDE;
    if constexpr (ring_ok<Tree, false>()) {
      v.fn[3] = &launch_eval_ring<Tree, M, PREC>;
      v.kernel[3] = (const void*)&k_eval_ring<Tree, M, PREC>;
      v.warp_bytes[3] = RingLayout<Tree, PREC, false>::STRIDE;
    }
    if constexpr (pair_eval_ok<Tree, M, PREC>()) {
      v.fn[4] = &launch_eval_pair<Tree>;
      v.kernel[4] = (const void*)&k_eval_pair<Tree>;
      v.warp_bytes[4] = PairEvalLayout<Tree>::STRIDE;
    }
    constexpr DefaultGeo g = default_geometry<Tree, M, PREC, false>();
    v.default_variant = g.variant;
    v.default_threads = g.threads;
    v.default_bps = g.bps;
  }
  register_eval(Sig<Tree>::str(), PREC, math, v, Vps<PREC>::value);
}

template <class Tree, class M>
void reg_adjoint(int math) {
  Variants v{};
  v.fn[0] = &launch_adjoint<Tree, M>;
  v.kernel[0] = (const void*)&k_adjoint<Tree, M>;
  v.fn[1] = &launch_adjoint_tma<Tree, M>;
  v.kernel[1] = (const void*)&k_adjoint_tma<Tree, M>;
  v.warp_bytes[1] = tma_warp_stride(TileBytes<Tree, P_F64, true>::value);
  v.fn[2] = &launch_adjoint_lazy<Tree, M>;
  v.kernel[2] = (const void*)&k_adjoint_lazy<Tree, M>;
  v.warp_bytes[2] = LazyLayout<Tree, P_F64, true>::STRIDE;
  if constexpr (ring_ok<Tree, true>()) {
    v.fn[3] = &launch_adjoint_ring<Tree, M>;
    v.kernel[3] = (const void*)&k_adjoint_ring<Tree, M>;
    v.warp_bytes[3] = RingLayout<Tree, P_F64, true>::STRIDE;
  }
  if constexpr (pair_adjoint_ok<Tree, M>()) {
    v.fn[4] = &launch_adjoint_pair<Tree>;
    v.kernel[4] = (const void*)&k_adjoint_pair<Tree>;
    v.warp_bytes[4] = PairAdjLayout::STRIDE;
  }
  constexpr DefaultGeo g = default_geometry<Tree, M, P_F64, true>();
  v.default_variant = g.variant;
  v.default_threads = g.threads;
  v.default_bps = g.bps;
  register_adjoint(Sig<Tree>::str(), math, v);
}

// ------------------------------------------------------------ catalogue
namespace cat {
using MM = Mul<LM<0>, LM<1>>;
using ScaleMM = Scale<0, Mul<LM<0>, LM<1>>>;
using AdjMM = Mul<Adj<LM<0>>, LM<1>>;
using MAdjM = Mul<LM<0>, Adj<LM<1>>>;
using AdjMAdjM = Mul<Adj<LM<0>>, Adj<LM<1>>>;
using Square = Mul<LM<0>, LM<0>>;
using MV = Mul<LM<0>, LV<1>>;
using AdjMV = Mul<Adj<LM<0>>, LV<1>>;
using MMV = Mul<Mul<LM<0>, LM<1>>, LV<2>>;
using E1 = Add<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>;
using E1Sub = Sub<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>;
using E1Lin = Add<Scale<0, Mul<LM<0>, LM<1>>>, Scale<1, Mul<LM<2>, LM<3>>>>;
using E2 = Add<Mul<Mul<LM<0>, LM<1>>, LM<2>>, Scale<0, LM<3>>>;
using MMM = Mul<Mul<LM<0>, LM<1>>, LM<2>>;
using E3 = Sub<Mul<Adj<LM<0>>, LM<1>>, Mul<LM<1>, Adj<LM<0>>>>;
using Comm = Sub<Mul<LM<0>, LM<1>>, Mul<LM<1>, LM<0>>>;
using CopyM = LM<0>;
using AdjM = Adj<LM<0>>;
using ScaleM = Scale<0, LM<0>>;
using AddM = Add<LM<0>, LM<1>>;
using SubM = Sub<LM<0>, LM<1>>;
using AxpyM = Add<Scale<0, LM<0>>, LM<1>>;
using CopyV = LV<0>;
using ScaleV = Scale<0, LV<0>>;
using AddV = Add<LV<0>, LV<1>>;
using SubV = Sub<LV<0>, LV<1>>;
using AxpyV = Add<Scale<0, LV<0>>, LV<1>>;
using CopyR = LR<0>;
using AddR = Add<LR<0>, LR<1>>;
using SubR = Sub<LR<0>, LR<1>>;
using MulR = Mul<LR<0>, LR<1>>;
using ScaleR = Scale<0, LR<0>>;
using L2R = Add<Add<LR<0>, LR<1>>, Mul<LR<0>, LR<1>>>;  // v1+v2+v1*v2 (Listing 2)
}  // namespace cat

}  // namespace su3s
