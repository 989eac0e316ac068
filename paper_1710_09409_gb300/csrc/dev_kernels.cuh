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

#include "dev_expr.cuh"
#include "dev_field.cuh"
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
    m[12 + 2 * c] = M::finish(re);
    m[12 + 2 * c + 1] = M::finish(im);
  }
}

// Load leaf slot I (kind K) of VPS consecutive sites starting at site s.
template <int K, int PREC, class M, int VPS, class C>
__device__ __forceinline__ void load_obj(const FieldDesc& f, int64_t s, int mu, C* ctx, int slot) {
  const int64_t b = elem_base(f, s, mu);
  if constexpr (K == KR) {
    static_assert(VPS == 1, "real fields are FP64");
    ctx[0].leaf[slot][0] = StoreReal::template load<M>(f.ptr, b);
  } else {
    using St = typename BaseStore<PREC>::type;
    constexpr int NC = (K == KV) ? 3 : (IsC12<PREC>::value ? 6 : 9);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      typename M::R re[VPS], im[VPS];
      St::template load<M>(f.ptr, b + c * f.s_c, re, im);
#pragma unroll
      for (int v = 0; v < VPS; ++v) {
        ctx[v].leaf[slot][2 * c] = re[v];
        ctx[v].leaf[slot][2 * c + 1] = im[v];
      }
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
template <class Tree, class M, int PREC>
__device__ __forceinline__ void eval_sites(const KParams& p, int64_t t, int mu) {
  constexpr int VPS = Vps<PREC>::value;
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int W = Width<Tree::kind>::value;
  Ctx<M, NL, NS> ctx[VPS];
#pragma unroll
  for (int v = 0; v < VPS; ++v)
#pragma unroll
    for (int k = 0; k < (NS > 0 ? NS : 1); ++k)
      ctx[v].sc[k] = M::scalar(p.sc[k], p.sch[k], p.scl[k]);
  const int64_t s = t * VPS;
  load_leaves<Tree, 0, PREC, M, VPS>(p, s, mu, ctx);
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

template <class Tree, class M, int PREC>
__global__ void __launch_bounds__(256) k_eval(const __grid_constant__ KParams p) {
  const int mu = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < p.nvec; t += stride)
    eval_sites<Tree, M, PREC>(p, t, mu);
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

template <class Tree, class M>
__global__ void __launch_bounds__(256) k_adjoint(const __grid_constant__ GParams p) {
  constexpr int NL = Tree::nleaf;
  constexpr int NS = Tree::nsc;
  constexpr int W = Width<Tree::kind>::value;
  const int mu = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.k.nvec; s += stride) {
    Ctx<M, NL, NS> ctx[1];
#pragma unroll
    for (int k = 0; k < (NS > 0 ? NS : 1); ++k)
      ctx[0].sc[k] = M::scalar(p.k.sc[k], p.k.sch[k], p.k.scl[k]);
    load_leaves<Tree, 0, P_F64, M, 1>(p.k, s, mu, ctx);
    // dL/dZ
    Ctx<M, 1, 0> g[1];
    load_obj<Tree::kind, P_F64, M, 1>(p.gout, s, mu, g, 0);
    GradAcc<M, NL> ga;
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int r = 0; r < 18; ++r) ga.g[i][r] = M::zero();
    GradSink<Tree, M> sink{&p, s, mu};
    Rev<Tree>::template run<Tree, M>(ctx[0], g[0].leaf[0], ga, sink);
    store_repeated<Tree, 0, M>(ga, sink);
    (void)W;
  }
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

// Registry hooks implemented by the library (api.cu).
void register_eval(const std::string& sig, int prec, int math, LaunchFn fn, const void* kernel,
                   int vps);
void register_adjoint(const std::string& sig, int math, LaunchFn fn, const void* kernel);

template <class Tree, class M, int PREC>
void reg_eval(int math) {
  register_eval(Sig<Tree>::str(), PREC, math, &launch_eval<Tree, M, PREC>,
                (const void*)&k_eval<Tree, M, PREC>, Vps<PREC>::value);
}

template <class Tree, class M>
void reg_adjoint(int math) {
  register_adjoint(Sig<Tree>::str(), math, &launch_adjoint<Tree, M>,
                   (const void*)&k_adjoint<Tree, M>);
}

// ------------------------------------------------------------ catalogue
namespace cat {
using MM = Mul<LM<0>, LM<1>>;
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
