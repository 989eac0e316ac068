// Compile-time expression trees evaluated per site in registers.
//
// The tree of an expression is a type, as in the expression-template engine
// of arXiv:1710.09409 (Sec. 3, Listing 1: LatticeBinaryExpression<Op,T1,T2>
// and eval(ss, expr)), but here a fixed catalogue of tree types is compiled
// ahead of time and a runtime tree is matched to one of them by its
// signature; leaf fields and real factors are runtime values.
//
//   LM<i>, LV<i>, LR<i>   leaf slot i holding a matrix / vector / real field
//   Mul<X,Y>              product (matrix*matrix, matrix*vector, real*real)
//   Add<X,Y>, Sub<X,Y>    sum, difference
//   Scale<k,X>            real factor number k times X
//   Adj<X>                Hermitian adjoint of a matrix
//
// Forward evaluation accumulates: the terms of sums and products of a node
// go straight into one accumulator per output real (so a*b + c*d is one
// 12-term dot product per output real, with no intermediate rounding), and an
// adjoint operand of a product is read transposed and conjugated in place.
// Reverse mode (Back) applies dA = G B^dagger, dB = A^dagger G and the chain
// rule through sums, factors and adjoints.
#pragma once

#include "dev_math.cuh"

namespace su3s {

enum { KM = 0, KV = 1, KR = 2 };

template <int K>
struct Width;
template <>
struct Width<KM> {
  static constexpr int value = 18;
};
template <>
struct Width<KV> {
  static constexpr int value = 6;
};
template <>
struct Width<KR> {
  static constexpr int value = 1;
};

template <int I>
struct LM {
  static constexpr int kind = KM, slot = I, nleaf = I + 1, nsc = 0;
  static constexpr bool is_leaf = true, accumulates = false;
};
template <int I>
struct LV {
  static constexpr int kind = KV, slot = I, nleaf = I + 1, nsc = 0;
  static constexpr bool is_leaf = true, accumulates = false;
};
template <int I>
struct LR {
  static constexpr int kind = KR, slot = I, nleaf = I + 1, nsc = 0;
  static constexpr bool is_leaf = true, accumulates = false;
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <class X, class Y>
struct Mul {
  static constexpr int kind = (X::kind == KM && Y::kind == KM)   ? KM
                              : (X::kind == KM && Y::kind == KV) ? KV
                              : (X::kind == KR && Y::kind == KR) ? KR
                                                                 : -1;
  static_assert(kind >= 0, "ill-typed product");
  static constexpr int nleaf = cmax(X::nleaf, Y::nleaf), nsc = cmax(X::nsc, Y::nsc);
  static constexpr bool is_leaf = false, accumulates = true;
};
template <class X, class Y>
struct Add {
  static_assert(X::kind == Y::kind, "ill-typed sum");
  static constexpr int kind = X::kind;
  static constexpr int nleaf = cmax(X::nleaf, Y::nleaf), nsc = cmax(X::nsc, Y::nsc);
  static constexpr bool is_leaf = false, accumulates = true;
};
template <class X, class Y>
struct Sub {
  static_assert(X::kind == Y::kind, "ill-typed difference");
  static constexpr int kind = X::kind;
  static constexpr int nleaf = cmax(X::nleaf, Y::nleaf), nsc = cmax(X::nsc, Y::nsc);
  static constexpr bool is_leaf = false, accumulates = true;
};
template <int K, class X>
struct Scale {
  static constexpr int kind = X::kind;
  static constexpr int nleaf = X::nleaf, nsc = cmax(X::nsc, K + 1);
  static constexpr bool is_leaf = false, accumulates = true;
};
template <class X>
struct Adj {
  static_assert(X::kind == KM, "adjoint of a non-matrix");
  static constexpr int kind = KM;
  static constexpr int nleaf = X::nleaf, nsc = X::nsc;
  static constexpr bool is_leaf = false, accumulates = false;
};

// Number of occurrences of leaf slot I in tree T.
template <class T, int I>
struct Count;
template <int J, int I>
struct Count<LM<J>, I> {
  static constexpr int value = (I == J);
};
template <int J, int I>
struct Count<LV<J>, I> {
  static constexpr int value = (I == J);
};
template <int J, int I>
struct Count<LR<J>, I> {
  static constexpr int value = (I == J);
};
template <class X, class Y, int I>
struct Count<Mul<X, Y>, I> {
  static constexpr int value = Count<X, I>::value + Count<Y, I>::value;
};
template <class X, class Y, int I>
struct Count<Add<X, Y>, I> {
  static constexpr int value = Count<X, I>::value + Count<Y, I>::value;
};
template <class X, class Y, int I>
struct Count<Sub<X, Y>, I> {
  static constexpr int value = Count<X, I>::value + Count<Y, I>::value;
};
template <int K, class X, int I>
struct Count<Scale<K, X>, I> {
  static constexpr int value = Count<X, I>::value;
};
template <class X, int I>
struct Count<Adj<X>, I> {
  static constexpr int value = Count<X, I>::value;
};

// Kind of leaf slot I in tree T (-1 if absent).
template <class T, int I>
struct LeafKind;
template <int J, int I>
struct LeafKind<LM<J>, I> {
  static constexpr int value = (I == J) ? KM : -1;
};
template <int J, int I>
struct LeafKind<LV<J>, I> {
  static constexpr int value = (I == J) ? KV : -1;
};
template <int J, int I>
struct LeafKind<LR<J>, I> {
  static constexpr int value = (I == J) ? KR : -1;
};
template <class X, class Y, int I>
struct LeafKind<Mul<X, Y>, I> {
  static constexpr int value = cmax(LeafKind<X, I>::value, LeafKind<Y, I>::value);
};
template <class X, class Y, int I>
struct LeafKind<Add<X, Y>, I> {
  static constexpr int value = cmax(LeafKind<X, I>::value, LeafKind<Y, I>::value);
};
template <class X, class Y, int I>
struct LeafKind<Sub<X, Y>, I> {
  static constexpr int value = cmax(LeafKind<X, I>::value, LeafKind<Y, I>::value);
};
template <int K, class X, int I>
struct LeafKind<Scale<K, X>, I> {
  static constexpr int value = LeafKind<X, I>::value;
};
template <class X, int I>
struct LeafKind<Adj<X>, I> {
  static constexpr int value = LeafKind<X, I>::value;
};

// Degree of tree T: the most factors (leaves and real factors) in one term of
// its expansion; it sets the range guard's bound (guard_hi).
template <class T>
struct Degree {
  static constexpr int value = 1;  // leaves
};
template <class X, class Y>
struct Degree<Mul<X, Y>> {
  static constexpr int value = Degree<X>::value + Degree<Y>::value;
};
template <class X, class Y>
struct Degree<Add<X, Y>> {
  static constexpr int value = cmax(Degree<X>::value, Degree<Y>::value);
};
template <class X, class Y>
struct Degree<Sub<X, Y>> {
  static constexpr int value = cmax(Degree<X>::value, Degree<Y>::value);
};
template <int K, class X>
struct Degree<Scale<K, X>> {
  static constexpr int value = Degree<X>::value + 1;
};
template <class X>
struct Degree<Adj<X>> {
  static constexpr int value = Degree<X>::value;
};

// Whether a site whose inputs' largest high word is g must be evaluated
// again in native FP64 (range guard of the FP64-accurate arithmetics; the
// reverse mode of T has T's degree, dL/dZ taking the place of one factor).
template <class T>
__device__ __forceinline__ bool guard_trips(uint32_t g) {
  return g >= guard_hi(Degree<T>::value);
}

// Operand view: Adj<B> is read as B with the adjoint flag set.
template <class T>
struct Operand {
  using base = T;
  static constexpr bool adj = false;
};
template <class B>
struct Operand<Adj<B>> {
  using base = B;
  static constexpr bool adj = true;
};

// Per-site evaluation context: loaded leaves and real factors.  Leaf values
// are reached through leaf_value<slot, W>() so that a context can also fetch
// them on demand (the TMA-staged kernels read a leaf from shared memory at its
// first use and refill its buffer after its last use).
template <class M, int NL, int NS>
struct Ctx {
  typename M::R leaf[NL][18];
  typename M::R sc[NS > 0 ? NS : 1];
  uint32_t gmax = 0;  // range guard: largest input high word read into this context
  template <int I, int W>
  __device__ __forceinline__ void leaf_value(typename M::R* out) const {
#pragma unroll
    for (int r = 0; r < W; ++r) out[r] = leaf[I][r];
  }
};

// ----------------------------------------------------------- primitives
// Packed form of a 3x3 complex product for the pair arithmetic: output (i,k)
// keeps (re, im) in the two lanes of one DAcc2.  Per inner index j, the terms
//   re += SG xr yr,             im += SG sy xr ym        (A: y = (yr, ym))
//   re += -SG sx sy xm ym,      im += SG sx xm yr        (B: y = (ym, yr))
// enter in the scalar order (A then B, j = 0, 1, 2), so each lane repeats
// MathDF's operations.  The signs ride on the x pairs, built once per element
// of x for the three outputs of its row; the A pairs of y are the loaded
// values themselves and only the swapped B pairs are extra registers.
template <bool FIRST, int SG, bool AX, bool AY>
__device__ __forceinline__ void mm_pairs(DAcc2* P, const df* x, const df* y) {
  constexpr int sx = AX ? -1 : 1, sy = AY ? -1 : 1;
  constexpr int ar = SG, ai = SG * sy, br = -SG * sx * sy, bi = SG * sx;
  df2 ya[9], yb[9];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int yi = AY ? (3 * k + j) : (3 * j + k);
      const df yr = y[2 * yi], ym = y[2 * yi + 1];
      ya[3 * j + k] = df2{make_float2(yr.h, ym.h), make_float2(yr.l, ym.l)};
      yb[3 * j + k] = df2{make_float2(ym.h, yr.h), make_float2(ym.l, yr.l)};
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int xi = AX ? (3 * j + i) : (3 * i + j);
      const df xr = x[2 * xi], xm = x[2 * xi + 1];
      const df2 xa{make_float2(ar > 0 ? xr.h : -xr.h, ai > 0 ? xr.h : -xr.h),
                   make_float2(ar > 0 ? xr.l : -xr.l, ai > 0 ? xr.l : -xr.l)};
      const df2 xb{make_float2(br > 0 ? xm.h : -xm.h, bi > 0 ? xm.h : -xm.h),
                   make_float2(br > 0 ? xm.l : -xm.l, bi > 0 ? xm.l : -xm.l)};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        DAcc2& a = P[3 * i + k];
        if (FIRST && j == 0) df2_first(a, xa, ya[3 * j + k]);
        else df2_fma(a, xa, ya[3 * j + k]);
        df2_fma(a, xb, yb[3 * j + k]);
      }
    }
}

// Operand pairs of mm_pairs for SG = +1: x element (i, j) of op(x) with the
// signs of the two terms, y element (j, k) of op(y) and its swapped copy.
template <bool AX, bool AY>
__device__ __forceinline__ df2 row_xa(const df* x, int i, int j) {
  constexpr int ai = AY ? -1 : 1;
  const int xi = AX ? (3 * j + i) : (3 * i + j);
  const df xr = x[2 * xi];
  return df2{make_float2(xr.h, ai > 0 ? xr.h : -xr.h), make_float2(xr.l, ai > 0 ? xr.l : -xr.l)};
}
template <bool AX, bool AY>
__device__ __forceinline__ df2 row_xb(const df* x, int i, int j) {
  constexpr int sx = AX ? -1 : 1, sy = AY ? -1 : 1;
  constexpr int br = -sx * sy, bi = sx;
  const int xi = AX ? (3 * j + i) : (3 * i + j);
  const df xm = x[2 * xi + 1];
  return df2{make_float2(br > 0 ? xm.h : -xm.h, bi > 0 ? xm.h : -xm.h),
             make_float2(br > 0 ? xm.l : -xm.l, bi > 0 ? xm.l : -xm.l)};
}
template <bool AY>
__device__ __forceinline__ df2 row_ya(const df* y, int j, int k) {
  const int yi = AY ? (3 * k + j) : (3 * j + k);
  const df yr = y[2 * yi], ym = y[2 * yi + 1];
  return df2{make_float2(yr.h, ym.h), make_float2(yr.l, ym.l)};
}
template <bool AY>
__device__ __forceinline__ df2 row_yb(const df* y, int j, int k) {
  const int yi = AY ? (3 * k + j) : (3 * j + k);
  const df yr = y[2 * yi], ym = y[2 * yi + 1];
  return df2{make_float2(ym.h, yr.h), make_float2(ym.l, yr.l)};
}

// Rows i of two products at once, P[k] = row i of op(x0) op(y0) and Q[k] = row i
// of op(x1) op(y1), their terms interleaved; each output receives mm_pairs'
// operations in mm_pairs' order.
template <bool AX0, bool AY0, bool AX1, bool AY1>
__device__ __forceinline__ void mm_pairs_row2(DAcc2* P, DAcc2* Q, const df* x0, const df* y0,
                                              const df* x1, const df* y1, int i) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const df2 xa0 = row_xa<AX0, AY0>(x0, i, j), xb0 = row_xb<AX0, AY0>(x0, i, j);
    const df2 xa1 = row_xa<AX1, AY1>(x1, i, j), xb1 = row_xb<AX1, AY1>(x1, i, j);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const df2 ya0 = row_ya<AY0>(y0, j, k), yb0 = row_yb<AY0>(y0, j, k);
      const df2 ya1 = row_ya<AY1>(y1, j, k), yb1 = row_yb<AY1>(y1, j, k);
      if (j == 0) {
        df2_first(P[k], xa0, ya0);
        df2_first(Q[k], xa1, ya1);
      } else {
        df2_fma(P[k], xa0, ya0);
        df2_fma(Q[k], xa1, ya1);
      }
      df2_fma(P[k], xb0, yb0);
      df2_fma(Q[k], xb1, yb1);
    }
  }
}

// z (+)= SG * op(x) * op(y), 3x3 complex; op = adjoint when AX / AY.
template <class M, bool FIRST, int SG, bool AX, bool AY>
__device__ __forceinline__ void mm_acc(typename M::A* z, const typename M::R* x,
                                       const typename M::R* y) {
  constexpr int sx = AX ? -1 : 1, sy = AY ? -1 : 1;
  if constexpr (M::kPaired) {
    DAcc2 P[9];
    if constexpr (!FIRST) {
#pragma unroll
      for (int e = 0; e < 9; ++e) P[e] = dacc2_get(z[2 * e], z[2 * e + 1]);
    }
    mm_pairs<FIRST, SG, AX, AY>(P, x, y);
#pragma unroll
    for (int e = 0; e < 9; ++e) dacc2_put(z[2 * e], z[2 * e + 1], P[e]);
  } else if constexpr (M::kScaled) {
    // integer multiply-adds have a long latency: advance the 18 independent
    // accumulators together, one inner index j at a time
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          typename M::A& re = z[2 * (3 * i + k)];
          typename M::A& im = z[2 * (3 * i + k) + 1];
          const int xi = AX ? (3 * j + i) : (3 * i + j);
          const int yi = AY ? (3 * k + j) : (3 * j + k);
          if (FIRST && j == 0) {
            M::template fma<true, SG>(re, x[2 * xi], y[2 * yi]);
            M::template fma<true, SG * sy>(im, x[2 * xi], y[2 * yi + 1]);
          } else {
            M::template fma<false, SG>(re, x[2 * xi], y[2 * yi]);
            M::template fma<false, SG * sy>(im, x[2 * xi], y[2 * yi + 1]);
          }
          M::template fma<false, -SG * sx * sy>(re, x[2 * xi + 1], y[2 * yi + 1]);
          M::template fma<false, SG * sx>(im, x[2 * xi + 1], y[2 * yi]);
        }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        typename M::A& re = z[2 * (3 * i + k)];
        typename M::A& im = z[2 * (3 * i + k) + 1];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int xi = AX ? (3 * j + i) : (3 * i + j);
          const int yi = AY ? (3 * k + j) : (3 * j + k);
          const typename M::R& xr = x[2 * xi];
          const typename M::R& xm = x[2 * xi + 1];
          const typename M::R& yr = y[2 * yi];
          const typename M::R& ym = y[2 * yi + 1];
          if (FIRST && j == 0) {
            M::template fma<true, SG>(re, xr, yr);
            M::template fma<true, SG * sy>(im, xr, ym);
          } else {
            M::template fma<false, SG>(re, xr, yr);
            M::template fma<false, SG * sy>(im, xr, ym);
          }
          M::template fma<false, -SG * sx * sy>(re, xm, ym);
          M::template fma<false, SG * sx>(im, xm, yr);
        }
      }
  }
}

// Packed form of op(x) * v for the pair arithmetic, as mm_pairs: output i
// keeps (re, im) in one DAcc2; per j the terms xr (vr, vm) and xm (vm, vr)
// enter in the scalar order with the signs on the x pairs.
template <bool FIRST, int SG, bool AX>
__device__ __forceinline__ void mv_pairs(DAcc2* P, const df* x, const df* v) {
  constexpr int sx = AX ? -1 : 1;
  constexpr int br = -SG * sx, bi = SG * sx;
  df2 va[3], vb[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const df vr = v[2 * j], vm = v[2 * j + 1];
    va[j] = df2{make_float2(vr.h, vm.h), make_float2(vr.l, vm.l)};
    vb[j] = df2{make_float2(vm.h, vr.h), make_float2(vm.l, vr.l)};
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int xi = AX ? (3 * j + i) : (3 * i + j);
      const df xr = x[2 * xi], xm = x[2 * xi + 1];
      const df2 xa{make_float2(SG > 0 ? xr.h : -xr.h, SG > 0 ? xr.h : -xr.h),
                   make_float2(SG > 0 ? xr.l : -xr.l, SG > 0 ? xr.l : -xr.l)};
      const df2 xb{make_float2(br > 0 ? xm.h : -xm.h, bi > 0 ? xm.h : -xm.h),
                   make_float2(br > 0 ? xm.l : -xm.l, bi > 0 ? xm.l : -xm.l)};
      if (FIRST && j == 0) df2_first(P[i], xa, va[j]);
      else df2_fma(P[i], xa, va[j]);
      df2_fma(P[i], xb, vb[j]);
    }
}

// z (+)= SG * op(x) * v, x 3x3, v 3-vector.
template <class M, bool FIRST, int SG, bool AX>
__device__ __forceinline__ void mv_acc(typename M::A* z, const typename M::R* x,
                                       const typename M::R* v) {
  constexpr int sx = AX ? -1 : 1;
  if constexpr (M::kPaired) {
    DAcc2 P[3];
    if constexpr (!FIRST) {
#pragma unroll
      for (int i = 0; i < 3; ++i) P[i] = dacc2_get(z[2 * i], z[2 * i + 1]);
    }
    mv_pairs<FIRST, SG, AX>(P, x, v);
#pragma unroll
    for (int i = 0; i < 3; ++i) dacc2_put(z[2 * i], z[2 * i + 1], P[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      typename M::A& re = z[2 * i];
      typename M::A& im = z[2 * i + 1];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int xi = AX ? (3 * j + i) : (3 * i + j);
        if (FIRST && j == 0) {
          M::template fma<true, SG>(re, x[2 * xi], v[2 * j]);
          M::template fma<true, SG>(im, x[2 * xi], v[2 * j + 1]);
        } else {
          M::template fma<false, SG>(re, x[2 * xi], v[2 * j]);
          M::template fma<false, SG>(im, x[2 * xi], v[2 * j + 1]);
        }
        M::template fma<false, -SG * sx>(re, x[2 * xi + 1], v[2 * j + 1]);
        M::template fma<false, SG * sx>(im, x[2 * xi + 1], v[2 * j]);
      }
    }
  }
}

// z (+)= SG * u * w^dagger (outer product of 3-vectors): z_ij = u_i conj(w_j).
template <class M, bool FIRST, int SG>
__device__ __forceinline__ void outer_acc(typename M::A* z, const typename M::R* u,
                                          const typename M::R* w) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      typename M::A& re = z[2 * (3 * i + j)];
      typename M::A& im = z[2 * (3 * i + j) + 1];
      M::template fma<FIRST, SG>(re, u[2 * i], w[2 * j]);
      M::template fma<false, SG>(re, u[2 * i + 1], w[2 * j + 1]);
      M::template fma<FIRST, SG>(im, u[2 * i + 1], w[2 * j]);
      M::template fma<false, -SG>(im, u[2 * i], w[2 * j + 1]);
    }
}

// z += SG * op(x) * op(y), each output accumulated on its own and then added
// to z exactly (the sum of two products keeps two independent accumulations
// per output, which halves the rounding error of the pair arithmetic's tail).
template <class M, int SG, bool AX, bool AY>
__device__ __forceinline__ void mm_combine(typename M::A* z, const typename M::R* x,
                                           const typename M::R* y) {
  constexpr int sx = AX ? -1 : 1, sy = AY ? -1 : 1;
  if constexpr (M::kPaired) {
    DAcc2 P[9];
    mm_pairs<true, 1, AX, AY>(P, x, y);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      DAcc2 a = dacc2_get(z[2 * e], z[2 * e + 1]);
      df2_combine<SG>(a, P[e]);
      dacc2_put(z[2 * e], z[2 * e + 1], a);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        typename M::A re, im;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int xi = AX ? (3 * j + i) : (3 * i + j);
          const int yi = AY ? (3 * k + j) : (3 * j + k);
          if (j == 0) {
            M::template fma<true, 1>(re, x[2 * xi], y[2 * yi]);
            M::template fma<true, sy>(im, x[2 * xi], y[2 * yi + 1]);
          } else {
            M::template fma<false, 1>(re, x[2 * xi], y[2 * yi]);
            M::template fma<false, sy>(im, x[2 * xi], y[2 * yi + 1]);
          }
          M::template fma<false, -sx * sy>(re, x[2 * xi + 1], y[2 * yi + 1]);
          M::template fma<false, sx>(im, x[2 * xi + 1], y[2 * yi]);
        }
        M::template combine<SG>(z[2 * (3 * i + k)], re);
        M::template combine<SG>(z[2 * (3 * i + k) + 1], im);
      }
  }
}

template <class M, int SG, bool AX>
__device__ __forceinline__ void mv_combine(typename M::A* z, const typename M::R* x,
                                           const typename M::R* v) {
  constexpr int sx = AX ? -1 : 1;
  if constexpr (M::kPaired) {
    DAcc2 P[3];
    mv_pairs<true, 1, AX>(P, x, v);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      DAcc2 a = dacc2_get(z[2 * i], z[2 * i + 1]);
      df2_combine<SG>(a, P[i]);
      dacc2_put(z[2 * i], z[2 * i + 1], a);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      typename M::A re, im;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int xi = AX ? (3 * j + i) : (3 * i + j);
        if (j == 0) {
          M::template fma<true, 1>(re, x[2 * xi], v[2 * j]);
          M::template fma<true, 1>(im, x[2 * xi], v[2 * j + 1]);
        } else {
          M::template fma<false, 1>(re, x[2 * xi], v[2 * j]);
          M::template fma<false, 1>(im, x[2 * xi], v[2 * j + 1]);
        }
        M::template fma<false, -sx>(re, x[2 * xi + 1], v[2 * j + 1]);
        M::template fma<false, sx>(im, x[2 * xi + 1], v[2 * j]);
      }
      M::template combine<SG>(z[2 * i], re);
      M::template combine<SG>(z[2 * i + 1], im);
    }
  }
}

template <class M, int W, bool FIRST, int SG>
__device__ __forceinline__ void vec_add(typename M::A* z, const typename M::R* x) {
#pragma unroll
  for (int r = 0; r < W; ++r) M::template add<FIRST, SG>(z[r], x[r]);
}

template <class M, int W, bool FIRST, int SG>
__device__ __forceinline__ void vec_scale_add(typename M::A* z, const typename M::R& s,
                                              const typename M::R* x) {
  if constexpr (M::kScaled && !FIRST) {
    // the product s*x has its own scale: form it, then align and add
#pragma unroll
    for (int r = 0; r < W; ++r) M::compact(z[r]);
#pragma unroll
    for (int r = 0; r < W; ++r) {
      typename M::A t;
      M::template fma<true, 1>(t, s, x[r]);
      M::template combine<SG>(z[r], t);
    }
  } else {
#pragma unroll
    for (int r = 0; r < W; ++r) M::template fma<FIRST, SG>(z[r], s, x[r]);
  }
}

template <class M>
__device__ __forceinline__ void adjoint(typename M::R* z, const typename M::R* x) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      z[2 * (3 * i + j)] = x[2 * (3 * j + i)];
      z[2 * (3 * i + j) + 1] = M::neg(x[2 * (3 * j + i) + 1]);
    }
}

// Accumulators of one object -> operand values (with a shared exponent for
// the fixed-point arithmetic).
template <class M, int W>
__device__ __forceinline__ void finish(typename M::R* z, const typename M::A* a) {
  if constexpr (M::kScaled) {
    M::template finish_obj<W>(z, a);
  } else {
#pragma unroll
    for (int r = 0; r < W; ++r) z[r] = M::finish(a[r]);
  }
}

// ------------------------------------------------------------ forward
// Value of node T (normalised) into out[Width].
template <class T, class M, class C>
__device__ __forceinline__ void value(const C& ctx, typename M::R* out);

// acc (+)= SG * value(T)
template <class T, class M, bool FIRST, int SG, class C>
__device__ __forceinline__ void acc_into(const C& ctx, typename M::A* acc);

// Leaves: copy from the context.
template <class T, class M, class C>
__device__ __forceinline__ void value(const C& ctx, typename M::R* out) {
  constexpr int W = Width<T::kind>::value;
  if constexpr (T::is_leaf) {
    ctx.template leaf_value<T::slot, W>(out);
  } else if constexpr (T::accumulates) {
    typename M::A a[W];
    acc_into<T, M, true, 1>(ctx, a);
    finish<M, W>(out, a);
  } else {  // Adj
    using X = typename Operand<T>::base;
    typename M::R x[18];
    value<X, M>(ctx, x);
    adjoint<M>(out, x);
  }
}

template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Mul<X, Y>*);
template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Add<X, Y>*);
template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Sub<X, Y>*);
template <class M, bool FIRST, int SG, class C, int K, class X>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Scale<K, X>*);

template <class T, class M, bool FIRST, int SG, class C>
__device__ __forceinline__ void acc_into(const C& ctx, typename M::A* acc) {
  constexpr int W = Width<T::kind>::value;
  if constexpr (!T::accumulates) {
    typename M::R v[W];
    value<T, M>(ctx, v);
    vec_add<M, W, FIRST, SG>(acc, v);
  } else {
    acc_node<M, FIRST, SG>(ctx, acc, (T*)nullptr);
  }
}

template <class M, int SG, class C, class X, class Y>
__device__ __forceinline__ void mul_combine(const C& ctx, typename M::A* acc, Mul<X, Y>*);

template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Mul<X, Y>*) {
  if constexpr (M::kScaled && !FIRST) {
    // a product added to an accumulator of another scale
    mul_combine<M, SG>(ctx, acc, (Mul<X, Y>*)nullptr);
    return;
  }
  using OX = Operand<X>;
  using OY = Operand<Y>;
  using BX = typename OX::base;
  using BY = typename OY::base;
  typename M::R xv[Width<BX::kind>::value];
  typename M::R yv[Width<BY::kind>::value];
  value<BX, M>(ctx, xv);
  value<BY, M>(ctx, yv);
  if constexpr (Mul<X, Y>::kind == KM) {
    mm_acc<M, FIRST, SG, OX::adj, OY::adj>(acc, xv, yv);
  } else if constexpr (Mul<X, Y>::kind == KV) {
    mv_acc<M, FIRST, SG, OX::adj>(acc, xv, yv);
  } else {
    M::template fma<FIRST, SG>(acc[0], xv[0], yv[0]);
  }
}

template <class T>
struct IsMulNode {
  static constexpr bool value = false;
};
template <class X, class Y>
struct IsMulNode<Mul<X, Y>> {
  static constexpr bool value = true;
};

// acc += SG * (product node), accumulated per output on its own and combined.
template <class M, int SG, class C, class X, class Y>
__device__ __forceinline__ void mul_combine(const C& ctx, typename M::A* acc, Mul<X, Y>*) {
  using OX = Operand<X>;
  using OY = Operand<Y>;
  using BX = typename OX::base;
  using BY = typename OY::base;
  if constexpr (M::kScaled) {
#pragma unroll
    for (int r = 0; r < Width<Mul<X, Y>::kind>::value; ++r) M::compact(acc[r]);
  }
  typename M::R xv[Width<BX::kind>::value];
  typename M::R yv[Width<BY::kind>::value];
  value<BX, M>(ctx, xv);
  value<BY, M>(ctx, yv);
  if constexpr (Mul<X, Y>::kind == KM) {
    mm_combine<M, SG, OX::adj, OY::adj>(acc, xv, yv);
  } else if constexpr (Mul<X, Y>::kind == KV) {
    mv_combine<M, SG, OX::adj>(acc, xv, yv);
  } else {
    typename M::A t;
    M::template fma<true, 1>(t, xv[0], yv[0]);
    M::template combine<SG>(acc[0], t);
  }
}

template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Add<X, Y>*) {
  acc_into<X, M, FIRST, SG>(ctx, acc);
  if constexpr (IsMulNode<Y>::value && (IsMulNode<X>::value || FIRST)) mul_combine<M, SG>(ctx, acc, (Y*)nullptr);
  else acc_into<Y, M, false, SG>(ctx, acc);
}

template <class M, bool FIRST, int SG, class C, class X, class Y>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Sub<X, Y>*) {
  acc_into<X, M, FIRST, SG>(ctx, acc);
  if constexpr (IsMulNode<Y>::value && (IsMulNode<X>::value || FIRST)) mul_combine<M, -SG>(ctx, acc, (Y*)nullptr);
  else acc_into<Y, M, false, -SG>(ctx, acc);
}

template <class M, bool FIRST, int SG, class C, int K, class X>
__device__ __forceinline__ void acc_node(const C& ctx, typename M::A* acc, Scale<K, X>*) {
  constexpr int W = Width<X::kind>::value;
  typename M::R v[W];
  value<X, M>(ctx, v);
  vec_scale_add<M, W, FIRST, SG>(acc, ctx.sc[K], v);
}

// ------------------------------------------------------------ reverse
// Gradient accumulators of leaves that occur more than once; leaves that occur
// once have their gradient complete when it is formed and are emitted at once
// through the sink.
template <class M, int NL>
struct GradAcc {
  typename M::A g[NL][18];
};

// gradient contribution for leaf slot I given as a ready accumulator
template <class M, int W, int I, bool ONCE, class GA, class Sink>
__device__ __forceinline__ void emit_acc(const typename M::A* contrib, GA& ga, Sink& sink) {
  if constexpr (ONCE) {
    sink.template put<I, W>(contrib);
  } else if constexpr (M::kScaled) {
#pragma unroll
    for (int r = 0; r < W; ++r) M::template combine<1>(ga.g[I][r], contrib[r]);
  } else {
#pragma unroll
    for (int r = 0; r < W; ++r) {
      typename M::R v = M::finish(contrib[r]);
      M::template add<false, 1>(ga.g[I][r], v);
    }
  }
}

// Tree-wide occurrence counts are needed at the leaves: carry the root type.
template <class Root>
struct Rev {
  template <class T, class M, class C, class GA, class Sink>
  __device__ static __forceinline__ void run(const C& ctx, const typename M::R* G, GA& ga,
                                             Sink& sink) {
    constexpr int W = Width<T::kind>::value;
    if constexpr (T::is_leaf) {
      typename M::A a[W];
      vec_add<M, W, true, 1>(a, G);
      emit_acc<M, W, T::slot, Count<Root, T::slot>::value == 1>(a, ga, sink);
    } else {
      node<M>(ctx, G, ga, sink, (T*)nullptr);
    }
  }

  // Feed a gradient that is a product (given as an accumulator-producing
  // lambda) into operand node T: directly for leaves, else through a value.
  template <class T, class M, class C, class GA, class Sink, class F>
  __device__ static __forceinline__ void feed(const C& ctx, GA& ga, Sink& sink, F&& make) {
    constexpr int W = Width<T::kind>::value;
    typename M::A a[W];
    make(a);
    if constexpr (T::is_leaf) {
      emit_acc<M, W, T::slot, Count<Root, T::slot>::value == 1>(a, ga, sink);
    } else {
      typename M::R v[W];
      finish<M, W>(v, a);
      run<T, M>(ctx, v, ga, sink);
    }
  }

  // Z = op(BX) op(BY).  The gradient of each operand needs G and the other
  // operand only, so the other operand is fetched just before its use: Y's
  // value, then d(BX); X's value, then d(BY).  One operand is live at a time.
  template <class M, class C, class GA, class Sink, class X, class Y>
  __device__ static __forceinline__ void node(const C& ctx, const typename M::R* G, GA& ga,
                                              Sink& sink, Mul<X, Y>*) {
    using OX = Operand<X>;
    using OY = Operand<Y>;
    using BX = typename OX::base;
    using BY = typename OY::base;
    constexpr bool ax = OX::adj, ay = OY::adj;
    {
      typename M::R yv[Width<BY::kind>::value];
      value<BY, M>(ctx, yv);
      if constexpr (Mul<X, Y>::kind == KM) {
        // d(base X): ax ? (Y G^dagger) : (G Y^dagger), with Y = op(BY)
        feed<BX, M>(ctx, ga, sink, [&](typename M::A* a) {
          if constexpr (ax) mm_acc<M, true, 1, ay, true>(a, yv, G);
          else mm_acc<M, true, 1, false, !ay>(a, G, yv);
        });
      } else if constexpr (Mul<X, Y>::kind == KV) {
        // Z = op(BX) v: d op(BX) = G v^dagger; d(BX) = ax ? v G^dagger : G v^dagger
        feed<BX, M>(ctx, ga, sink, [&](typename M::A* a) {
          if constexpr (ax) outer_acc<M, true, 1>(a, yv, G);
          else outer_acc<M, true, 1>(a, G, yv);
        });
      } else {
        feed<BX, M>(ctx, ga, sink,
                    [&](typename M::A* a) { M::template fma<true, 1>(a[0], G[0], yv[0]); });
      }
    }
    {
      typename M::R xv[Width<BX::kind>::value];
      value<BX, M>(ctx, xv);
      if constexpr (Mul<X, Y>::kind == KM) {
        // d(base Y): ay ? (G^dagger X) : (X^dagger G), with X = op(BX)
        feed<BY, M>(ctx, ga, sink, [&](typename M::A* a) {
          if constexpr (ay) mm_acc<M, true, 1, true, ax>(a, G, xv);
          else mm_acc<M, true, 1, !ax, false>(a, xv, G);
        });
      } else if constexpr (Mul<X, Y>::kind == KV) {
        // dv = op(BX)^dagger G
        feed<BY, M>(ctx, ga, sink, [&](typename M::A* a) { mv_acc<M, true, 1, !ax>(a, xv, G); });
      } else {
        feed<BY, M>(ctx, ga, sink,
                    [&](typename M::A* a) { M::template fma<true, 1>(a[0], xv[0], G[0]); });
      }
    }
  }

  template <class M, class C, class GA, class Sink, class X, class Y>
  __device__ static __forceinline__ void node(const C& ctx, const typename M::R* G, GA& ga,
                                              Sink& sink, Add<X, Y>*) {
    run<X, M>(ctx, G, ga, sink);
    run<Y, M>(ctx, G, ga, sink);
  }

  template <class M, class C, class GA, class Sink, class X, class Y>
  __device__ static __forceinline__ void node(const C& ctx, const typename M::R* G, GA& ga,
                                              Sink& sink, Sub<X, Y>*) {
    constexpr int W = Width<X::kind>::value;
    run<X, M>(ctx, G, ga, sink);
    typename M::R ng[W];
#pragma unroll
    for (int r = 0; r < W; ++r) ng[r] = M::neg(G[r]);
    run<Y, M>(ctx, ng, ga, sink);
  }

  template <class M, class C, class GA, class Sink, int K, class X>
  __device__ static __forceinline__ void node(const C& ctx, const typename M::R* G, GA& ga,
                                              Sink& sink, Scale<K, X>*) {
    constexpr int W = Width<X::kind>::value;
    feed<X, M>(ctx, ga, sink,
               [&](typename M::A* a) { vec_scale_add<M, W, true, 1>(a, ctx.sc[K], G); });
  }

  template <class M, class C, class GA, class Sink, class X>
  __device__ static __forceinline__ void node(const C& ctx, const typename M::R* G, GA& ga,
                                              Sink& sink, Adj<X>*) {
    typename M::R g[18];
    adjoint<M>(g, G);
    run<X, M>(ctx, g, ga, sink);
  }
};

}  // namespace su3s
