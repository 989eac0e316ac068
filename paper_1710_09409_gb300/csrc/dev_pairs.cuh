// Two sites per lane for the pair arithmetic (MathDF): a warp takes two
// 32-site tiles at a time and lane t computes site t of both, every FP32
// operation of MathDF issued as one packed f32x2 instruction whose two lanes
// are the two sites (the one-pass evaluation of Sec. 3, Listing 1, over the
// vector of sites of Sec. 5, two sites per SIMD lane).
//
// The (re, im) packing of mm_pairs pairs the real and imaginary parts of one
// output, which needs every x element duplicated and every y element swapped
// into extra registers.  Here the two lanes always hold the same real of two
// sites, so the split FP64 inputs are the operands as they stand, and a
// term's sign is a compile-time choice between the addition and subtraction
// forms of TwoSum: no operand is copied, swapped or negated.  Each lane
// performs MathDF's scalar operations in MathDF's order (for every output,
// its terms in the order of mm_acc), so the results equal the other data
// movements' bit for bit.
//
// Operands are read from the staged tiles as the products need them, each
// element of a leaf once, so two sites fit the register file: forward
// products run in outer-product order (step j reads column j of op(X) and
// row j of op(Y) and updates all nine outputs); the reverse mode keeps dL/dZ
// in registers and runs each gradient one output row or column at a time.
//
// Included by dev_kernels.cuh (uses its staging, fallback and store helpers).
#pragma once

namespace su3s {

// one real of the two sites: leading and trailing FP32 parts, lane k = site k
using dp = df2;
// accumulator of one real of the two sites (MathDF's DAcc, lane-wise)
using dpa = DAcc2;

// df_split_bits of two FP64 values (the same real of the two sites).
__device__ __forceinline__ dp dp_split(uint32_t lo0, uint32_t hi0, uint32_t lo1, uint32_t hi1) {
  return df2_split(lo0, hi0, lo1, hi1);
}

// df_to_double of both lanes.
__device__ __forceinline__ void dp_to_double(const dpa& a, double& d0, double& d1) {
  df2_to_double(a, d0, d1);
}

__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a = +x*y (NEG: -x*y), MathDF::fma with FIRST.  With x negated every value of
// the sequence is the exact negation of the positive one (round to nearest
// even is symmetric), so the negative form negates the two results.  Zeros
// are the exception (the leading product's +0 addend turns a -0 product into
// +0): a result may differ from MathDF's in the sign of a zero, never in value.
template <bool NEG>
__device__ __forceinline__ void dp_first(dpa& a, const dp& x, const dp& y) {
  const float2 p = f2_mul_lead(x.h, y.h);
  const float2 np = f2_neg(p);
  float2 q = f2_fma(x.h, y.h, np);  // exact error of the leading product
  q = f2_fma(x.h, y.l, q);
  q = f2_fma(x.l, y.h, q);
  if (NEG) {
    a.S = np;
    a.lo = f2_neg(q);
  } else {
    a.S = p;
    a.lo = q;
  }
}

// a += x*y (NEG: a -= x*y), MathDF::fma without FIRST, lane-wise.  The
// negative form is MathDF's sequence for -x written with x: s = S - p, the
// error terms come out negated (c = -db, u = -t) and enter by subtraction
// (equal values; the sign of a zero may differ, as in dp_first).
template <bool NEG>
__device__ __forceinline__ void dp_fma(dpa& a, const dp& x, const dp& y) {
  const float2 p = f2_mul_lead(x.h, y.h);
  if (!NEG) {
    const float2 s = f2_add(a.S, p);        // TwoSum(S, xh*yh)
    const float2 nbp = f2_sub(a.S, s);      // -bp
    const float2 ap = f2_add(s, nbp);       // s - bp
    const float2 db = f2_fma(x.h, y.h, nbp);
    const float2 da = f2_sub(a.S, ap);
    float2 t = f2_add(da, db);
    t = f2_fma(x.l, y.h, t);
    t = f2_fma(x.h, y.l, t);
    a.S = s;
    a.lo = f2_add(a.lo, t);
  } else {
    const float2 s = f2_sub(a.S, p);        // TwoSum(S, -xh*yh)
    const float2 bp = f2_sub(s, a.S);
    const float2 ap = f2_sub(s, bp);
    const float2 c = f2_fma(x.h, y.h, bp);  // -db
    const float2 da = f2_sub(a.S, ap);
    float2 u = f2_sub(c, da);               // -(da + db)
    u = f2_fma(x.l, y.h, u);
    u = f2_fma(x.h, y.l, u);
    a.S = s;
    a.lo = f2_sub(a.lo, u);
  }
}

// One complex term of SG * op(X) op(Y) into output (re, im): x = (xr, xm) and
// y = (yr, ym) are the stored elements, op = adjoint when AX / AY.  The four
// real terms enter in mm_acc's order: xr yr, xr ym, then xm ym, xm yr.
template <bool FIRST, int SG, bool AX, bool AY>
__device__ __forceinline__ void dp_cterm(dpa& re, dpa& im, const dp& xr, const dp& xm,
                                         const dp& yr, const dp& ym) {
  constexpr int sx = AX ? -1 : 1, sy = AY ? -1 : 1;
  if constexpr (FIRST) {
    dp_first<(SG < 0)>(re, xr, yr);
    dp_first<(SG * sy < 0)>(im, xr, ym);
  } else {
    dp_fma<(SG < 0)>(re, xr, yr);
    dp_fma<(SG * sy < 0)>(im, xr, ym);
  }
  dp_fma<(-SG * sx * sy < 0)>(re, xm, ym);
  dp_fma<(SG * sx < 0)>(im, xm, yr);
}

// ------------------------------------------------------- operand sources
// A staged matrix object of both tiles: element e of this lane's sites, read
// from shared memory and split when fetched; the range guard takes its words.
struct PairStaged {
  const unsigned char* t0;  // the object's tile of the unit's first 32 sites
  const unsigned char* t1;  // ... of the second
  int lane;
  __device__ __forceinline__ void fetch(int e, dp& re, dp& im, uint32_t& g) const {
    const uint4 v0 = reinterpret_cast<const uint4*>(t0 + e * 512)[lane];
    const uint4 v1 = reinterpret_cast<const uint4*>(t1 + e * 512)[lane];
    g = guard_max(guard_max(g, v0.y, v0.w), v1.y, v1.w);
    re = dp_split(v0.x, v0.y, v1.x, v1.y);
    im = dp_split(v0.z, v0.w, v1.z, v1.w);
  }
  // the range guard of an object whose values are not needed (every input of
  // a site is checked, used or not)
  __device__ __forceinline__ void guard(uint32_t& g) const {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const uint4 v0 = reinterpret_cast<const uint4*>(t0 + e * 512)[lane];
      const uint4 v1 = reinterpret_cast<const uint4*>(t1 + e * 512)[lane];
      g = guard_max(guard_max(g, v0.y, v0.w), v1.y, v1.w);
    }
  }
};
// An object already split into registers (18 reals).
struct PairHeld {
  const dp* v;
  __device__ __forceinline__ void fetch(int e, dp& re, dp& im, uint32_t&) const {
    re = v[2 * e];
    im = v[2 * e + 1];
  }
};

// Step J of SG * op(X) op(Y) in outer-product order into all nine outputs
// acc[18]: column J of op(X) times row J of op(Y).
template <bool FIRST, int SG, bool AX, bool AY, class SX, class SY>
__device__ __forceinline__ void dp_mm_step(int J, dpa* acc, const SX& X, const SY& Y, uint32_t& g) {
  dp x[6], y[6];
#pragma unroll
  for (int i = 0; i < 3; ++i) X.fetch(AX ? (3 * J + i) : (3 * i + J), x[2 * i], x[2 * i + 1], g);
#pragma unroll
  for (int k = 0; k < 3; ++k) Y.fetch(AY ? (3 * k + J) : (3 * J + k), y[2 * k], y[2 * k + 1], g);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      dp_cterm<FIRST, SG, AX, AY>(acc[2 * (3 * i + k)], acc[2 * (3 * i + k) + 1],
                                            x[2 * i], x[2 * i + 1], y[2 * k], y[2 * k + 1]);
}

template <bool FIRST, int SG, bool AX, bool AY, class SX, class SY>
__device__ __forceinline__ void dp_mm(dpa* acc, const SX& X, const SY& Y, uint32_t& g) {
  dp_mm_step<FIRST, SG, AX, AY>(0, acc, X, Y, g);
  // steps 1 and 2 share one copy of the code (instruction cache)
#pragma unroll 1
  for (int j = 1; j < 3; ++j) dp_mm_step<false, SG, AX, AY>(j, acc, X, Y, g);
}

// Row I of op(X) op(Y) into acc[6] (outputs (I, 0..2)): row I of op(X) is
// fetched, op(Y) is held (I may vary at run time: only the fetch depends on it).
template <bool AX, bool AY, class SX>
__device__ __forceinline__ void dp_mm_row(int I, dpa* acc, const SX& X, const dp* y, uint32_t& g) {
  dp x[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) X.fetch(AX ? (3 * j + I) : (3 * I + j), x[2 * j], x[2 * j + 1], g);
  PairHeld Y{y};
  uint32_t none = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dp yr, ym;
      Y.fetch(AY ? (3 * k + j) : (3 * j + k), yr, ym, none);
      if (j == 0) dp_cterm<true, 1, AX, AY>(acc[2 * k], acc[2 * k + 1], x[2 * j], x[2 * j + 1], yr, ym);
      else dp_cterm<false, 1, AX, AY>(acc[2 * k], acc[2 * k + 1], x[2 * j], x[2 * j + 1], yr, ym);
    }
}

// Column K of op(X) op(Y) into acc[6] (outputs (0..2, K)): op(X) is held,
// column K of op(Y) is fetched.
template <bool AX, bool AY, class SY>
__device__ __forceinline__ void dp_mm_col(int K, dpa* acc, const dp* x, const SY& Y, uint32_t& g) {
  dp y[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) Y.fetch(AY ? (3 * K + j) : (3 * j + K), y[2 * j], y[2 * j + 1], g);
  PairHeld X{x};
  uint32_t none = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dp xr, xm;
      X.fetch(AX ? (3 * j + i) : (3 * i + j), xr, xm, none);
      if (j == 0) dp_cterm<true, 1, AX, AY>(acc[2 * i], acc[2 * i + 1], xr, xm, y[2 * j], y[2 * j + 1]);
      else dp_cterm<false, 1, AX, AY>(acc[2 * i], acc[2 * i + 1], xr, xm, y[2 * j], y[2 * j + 1]);
    }
}

// ----------------------------------------------------------- tree shapes
// Operands: a matrix leaf or its adjoint.
template <class T>
struct PairOp {
  static constexpr bool ok = false;
  static constexpr int slot = 0;
  static constexpr bool adj = false;
};
template <int I>
struct PairOp<LM<I>> {
  static constexpr bool ok = true;
  static constexpr int slot = I;
  static constexpr bool adj = false;
};
template <int I>
struct PairOp<Adj<LM<I>>> {
  static constexpr bool ok = true;
  static constexpr int slot = I;
  static constexpr bool adj = true;
};

// A product of two distinct matrix leaves (either may be an adjoint).
template <class T>
struct PairProd {
  static constexpr bool ok = false;
};
template <class X, class Y>
struct PairProd<Mul<X, Y>> {
  using OX = PairOp<X>;
  using OY = PairOp<Y>;
  static constexpr bool ok = OX::ok && OY::ok && OX::slot != OY::slot;
};

// Forward trees: one such product, or the sum or difference of two over four
// distinct leaves (every leaf element is read once).  P0, P1: the products;
// S1: the second one's sign.
template <class T>
struct PairShape {
  static constexpr bool ok = PairProd<T>::ok;
  static constexpr int nprod = 1;
  using P0 = T;
  using P1 = T;
  static constexpr int S1 = 1;
};
template <class X, class Y>
constexpr bool pair_disjoint() {
  if constexpr (PairProd<X>::ok && PairProd<Y>::ok) {
    using A = PairProd<X>;
    using B = PairProd<Y>;
    return A::OX::slot != B::OX::slot && A::OX::slot != B::OY::slot &&
           A::OY::slot != B::OX::slot && A::OY::slot != B::OY::slot;
  } else {
    return false;
  }
}
template <class X, class Y, int SG>
struct PairSum {
  static constexpr bool ok = pair_disjoint<X, Y>();
  static constexpr int nprod = 2;
  using P0 = X;
  using P1 = Y;
  static constexpr int S1 = SG;
};
template <class X, class Y>
struct PairShape<Add<X, Y>> : PairSum<X, Y, 1> {};
template <class X, class Y>
struct PairShape<Sub<X, Y>> : PairSum<X, Y, -1> {};

template <class Tree, class M, int PREC>
constexpr bool pair_eval_ok() {
  return std::is_same<M, MathDF>::value && PREC == P_F64 && Tree::kind == KM &&
         PairShape<Tree>::ok;
}
// Reverse mode: one product of two distinct matrix leaves.
template <class Tree, class M>
constexpr bool pair_adjoint_ok() {
  return std::is_same<M, MathDF>::value && Tree::kind == KM && PairProd<Tree>::ok;
}

// ------------------------------------------------------------ staging
constexpr int kPairObj = StageBytes<KM, P_F64>::value;  // one 32-site tile of a matrix

__host__ __device__ constexpr int pair_warp_stride(int data_bytes, int nbar) {
  return (data_bytes + 8 * nbar + 127) / 128 * 128;
}

// A unit whose second tile is past the end reads zeros there (stores of that
// tile are skipped): the warp clears the buffer with plain stores.  Its last
// tensor copy landed before the warp read it, and no copy into it is pending.
__device__ __forceinline__ void pair_zero(unsigned char* dst, int lane) {
  for (int o = lane * 16; o < kPairObj; o += 32 * 16)
    *reinterpret_cast<uint4*>(dst + o) = make_uint4(0u, 0u, 0u, 0u);
}

// Issue the tensor copies of one object of the unit starting at tile t0 (the
// second tile when has1) into dst (two tiles).
__device__ __forceinline__ void pair_issue_obj(const FieldDesc& f, const CUtensorMap* tm, int64_t t0,
                                               bool has1, int mu, unsigned char* dst,
                                               uint64_t* bar) {
  issue_obj<KM, P_F64>(f, tm, t0 << 5, mu, dst, bar);
  if (has1) issue_obj<KM, P_F64>(f, tm, (t0 + 1) << 5, mu, dst + kPairObj, bar);
}

__device__ __forceinline__ void pair_store_c(char* base, int64_t e0, int64_t e1, bool has1,
                                             const dpa& re, const dpa& im) {
  double r0, r1, i0, i1;
  dp_to_double(re, r0, r1);
  dp_to_double(im, i0, i1);
  st16(base + e0 * 16, make_uint4((uint32_t)__double2loint(r0), (uint32_t)__double2hiint(r0),
                                  (uint32_t)__double2loint(i0), (uint32_t)__double2hiint(i0)));
  if (has1) {
    st16(base + e1 * 16, make_uint4((uint32_t)__double2loint(r1), (uint32_t)__double2hiint(r1),
                                    (uint32_t)__double2loint(i1), (uint32_t)__double2hiint(i1)));
  }
}

// ------------------------------------------------------------ forward
// Buffers per warp: each leaf's object of both tiles, slot by slot, then one
// barrier per product; a product's leaves are refilled for the warp's next
// unit as soon as the product has read them.
template <class Tree>
struct PairEvalLayout {
  static constexpr int NL = Tree::nleaf;
  static constexpr int NP = PairShape<Tree>::nprod;
  static constexpr int DATA = NL * 2 * kPairObj;
  static constexpr int STRIDE = pair_warp_stride(DATA, NP);
};

template <class P>
__device__ __forceinline__ void pair_issue_prod(int lane, const KParams& p, int64_t t0,
                                                int64_t ntiles, int mu, unsigned char* buf,
                                                uint64_t* bar) {
  constexpr int SX = PairProd<P>::OX::slot, SY = PairProd<P>::OY::slot;
  if (lane == 0) {
    const bool has1 = t0 + 1 < ntiles;
    mbar_arrive_expect_tx(bar, (has1 ? 4 : 2) * kPairObj);
    pair_issue_obj(p.leaf[SX], &p.tm[SX], t0, has1, mu, buf + SX * 2 * kPairObj, bar);
    pair_issue_obj(p.leaf[SY], &p.tm[SY], t0, has1, mu, buf + SY * 2 * kPairObj, bar);
  }
  __syncwarp();
}

// acc (+)= SG * product P of this unit, its leaves read from the staged tiles.
template <class P, bool FIRST, int SG>
__device__ __forceinline__ void pair_prod(dpa* acc, const unsigned char* buf, int lane,
                                          uint32_t& g) {
  using OX = typename PairProd<P>::OX;
  using OY = typename PairProd<P>::OY;
  const PairStaged X{buf + OX::slot * 2 * kPairObj, buf + OX::slot * 2 * kPairObj + kPairObj, lane};
  const PairStaged Y{buf + OY::slot * 2 * kPairObj, buf + OY::slot * 2 * kPairObj + kPairObj, lane};
  dp_mm<FIRST, SG, OX::adj, OY::adj>(acc, X, Y, g);
}

template <class Tree>
__global__ void __launch_bounds__(256) k_eval_pair(const __grid_constant__ KParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.err)) return;
  using L = PairEvalLayout<Tree>;
  using S = PairShape<Tree>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = smem + warp * L::STRIDE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(buf + L::DATA);
  const int mu = blockIdx.y;
  const int64_t ntiles = p.nvec >> 5;
  const Range rg = warp_range((ntiles + 1) >> 1);  // units of two tiles
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < L::NP; ++i) mbar_init(&bars[i], 1);
    fence_barrier_init();
  }
  __syncwarp();
  int64_t u = rg.first;
  if (u < rg.end) {
    pair_issue_prod<typename S::P0>(lane, p, 2 * u, ntiles, mu, buf, &bars[0]);
    if constexpr (L::NP == 2) pair_issue_prod<typename S::P1>(lane, p, 2 * u, ntiles, mu, buf, &bars[1]);
  }
  uint32_t phase = 0;
  while (u < rg.end) {
    const int64_t t0 = 2 * u;
    const bool has1 = t0 + 1 < ntiles;
    if (!has1) {
#pragma unroll
      for (int i = 0; i < L::NL; ++i) pair_zero(buf + (2 * i + 1) * kPairObj, lane);
      __syncwarp();
    }
    const int64_t un = u + rg.stride;
    uint32_t g = p.gscal;
    dpa acc[18];
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[0], phase))) {
      if (lane == 0) report_timeout(p.err, &bars[0], phase);
      if constexpr (L::NP == 2) mbar_wait_bounded(&bars[1], phase);  // the other copies (bounded)
      break;
    }
    pair_prod<typename S::P0, true, 1>(acc, buf, lane, g);
    fence_proxy_async_smem();
    __syncwarp();
    if (un < rg.end) pair_issue_prod<typename S::P0>(lane, p, 2 * un, ntiles, mu, buf, &bars[0]);
    if constexpr (L::NP == 2) {
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[1], phase))) {
        if (lane == 0) report_timeout(p.err, &bars[1], phase);
        if (un < rg.end) mbar_wait_bounded(&bars[0], phase ^ 1);
        break;
      }
      // the second product has accumulators of its own, combined once at the
      // end (as mul_combine: fewer roundings of each 12-term output's tail)
      dpa acc1[18];
      pair_prod<typename S::P1, true, 1>(acc1, buf, lane, g);
      fence_proxy_async_smem();
      __syncwarp();
      if (un < rg.end) pair_issue_prod<typename S::P1>(lane, p, 2 * un, ntiles, mu, buf, &bars[1]);
#pragma unroll
      for (int e = 0; e < 18; ++e) df2_combine<S::S1>(acc[e], acc1[e]);
    }
    phase ^= 1;
    const int64_t s0 = (t0 << 5) + lane;
    if (__any_sync(0xffffffffu, guard_trips<Tree>(g))) {
      // a unit with a site out of range runs its sites in native FP64 (nothing
      // of it is stored yet, so in-place evaluation stays correct)
      eval_site_f64<Tree, P_F64>(p, s0, mu);
      if (has1) eval_site_f64<Tree, P_F64>(p, s0 + 32, mu);
    } else {
      const int64_t e0 = elem_base(p.dst, s0, mu), e1 = elem_base(p.dst, s0 + 32, mu);
      char* base = static_cast<char*>(p.dst.ptr);
#pragma unroll
      for (int c = 0; c < 9; ++c)
        pair_store_c(base, e0 + c * p.dst.s_c, e1 + c * p.dst.s_c, has1, acc[2 * c], acc[2 * c + 1]);
    }
    u = un;
  }
}

// ------------------------------------------------------------ reverse mode
// Z = op(BX) op(BY), distinct leaves.  dL/dZ (G) is read into registers at
// the start of a unit; d(BX) then reads BY, and d(BY) reads BX, from the
// staged tiles, each element once, one output row or column at a time:
//   d(BX) = ax ? op(BY) G^dagger : G op(BY)^dagger,
//   d(BY) = ay ? G^dagger op(BX) : op(BX)^dagger G   (as the fused kernels).
// Buffers per warp: G and BY of both tiles behind one barrier, refilled for
// the warp's next unit after d(BX); BX behind a second, refilled after d(BY).
struct PairAdjLayout {
  static constexpr int R0 = 4 * kPairObj;  // G t0, G t1, BY t0, BY t1
  static constexpr int R1 = 2 * kPairObj;  // BX t0, BX t1
  static constexpr int STRIDE = pair_warp_stride(R0 + R1, 2);
};

template <class Tree>
__device__ __forceinline__ void pair_issue_adj(int lane, const GParams& p, int64_t t0,
                                               int64_t ntiles, int mu, unsigned char* buf,
                                               uint64_t* bars, int group) {
  constexpr int SX = PairProd<Tree>::OX::slot, SY = PairProd<Tree>::OY::slot;
  if (lane == 0) {
    const bool has1 = t0 + 1 < ntiles;
    const int n = has1 ? 2 : 1;
    if (group == 0) {
      mbar_arrive_expect_tx(&bars[0], 2 * n * kPairObj);
      pair_issue_obj(p.gout, &p.tm_gout, t0, has1, mu, buf, &bars[0]);
      pair_issue_obj(p.k.leaf[SY], &p.k.tm[SY], t0, has1, mu, buf + 2 * kPairObj, &bars[0]);
    } else {
      mbar_arrive_expect_tx(&bars[1], n * kPairObj);
      pair_issue_obj(p.k.leaf[SX], &p.k.tm[SX], t0, has1, mu, buf + PairAdjLayout::R0, &bars[1]);
    }
  }
  __syncwarp();
}

// Gradient of one operand, G held, the other operand V staged.  GX: d(BX).
template <bool GX, bool ax, bool ay>
__device__ __forceinline__ void pair_grad_part(int R, const FieldDesc& f, int64_t e0, int64_t e1,
                                               bool has1, const dp* G, const PairStaged& V,
                                               uint32_t& g) {
  dpa acc[6];
  // rows where G is the right factor, columns where it is the left one
  constexpr bool by_row = GX ? ax : !ay;
  if constexpr (GX) {
    if constexpr (ax) dp_mm_row<ay, true>(R, acc, V, G, g);
    else dp_mm_col<false, !ay>(R, acc, G, V, g);
  } else {
    if constexpr (ay) dp_mm_col<true, ax>(R, acc, G, V, g);
    else dp_mm_row<!ax, false>(R, acc, V, G, g);
  }
  char* base = static_cast<char*>(f.ptr);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int64_t c = (by_row ? 3 * R + q : 3 * q + R) * f.s_c;
    pair_store_c(base, e0 + c, e1 + c, has1, acc[2 * q], acc[2 * q + 1]);
  }
}

template <bool GX, bool ax, bool ay>
__device__ __forceinline__ void pair_grad(const FieldDesc& f, int64_t s0, int mu, bool has1,
                                          const dp* G, const PairStaged& V, uint32_t& g) {
  const int64_t e0 = elem_base(f, s0, mu), e1 = elem_base(f, s0 + 32, mu);
  // a rolled loop: the three rows (columns) share one copy of the code, which
  // keeps the kernel within the instruction cache
#pragma unroll 1
  for (int r = 0; r < 3; ++r) pair_grad_part<GX, ax, ay>(r, f, e0, e1, has1, G, V, g);
}

// Read G of both tiles into registers (18 reals).
__device__ __forceinline__ void pair_hold(const PairStaged& s, dp* out, uint32_t& g) {
#pragma unroll
  for (int e = 0; e < 9; ++e) s.fetch(e, out[2 * e], out[2 * e + 1], g);
}

template <class Tree>
__global__ void __launch_bounds__(256) k_adjoint_pair(const __grid_constant__ GParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (!smem_aligned(smem, p.k.err)) return;
  using L = PairAdjLayout;
  using OX = typename PairProd<Tree>::OX;
  using OY = typename PairProd<Tree>::OY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = smem + warp * L::STRIDE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(buf + L::R0 + L::R1);
  const int mu = blockIdx.y;
  const int64_t ntiles = p.k.nvec >> 5;
  const Range rg = warp_range((ntiles + 1) >> 1);
  const FieldDesc& fx = p.gleaf[OX::slot];
  const FieldDesc& fy = p.gleaf[OY::slot];
  if (lane == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  __syncwarp();
  int64_t u = rg.first;
  if (u < rg.end) {
    pair_issue_adj<Tree>(lane, p, 2 * u, ntiles, mu, buf, bars, 0);
    pair_issue_adj<Tree>(lane, p, 2 * u, ntiles, mu, buf, bars, 1);
  }
  const PairStaged SG_{buf, buf + kPairObj, lane};
  const PairStaged SBY{buf + 2 * kPairObj, buf + 3 * kPairObj, lane};
  const PairStaged SBX{buf + L::R0, buf + L::R0 + kPairObj, lane};
  uint32_t phase = 0;
  while (u < rg.end) {
    const int64_t t0 = 2 * u;
    const bool has1 = t0 + 1 < ntiles;
    if (!has1) {
      pair_zero(buf + kPairObj, lane);
      pair_zero(buf + 3 * kPairObj, lane);
      pair_zero(buf + L::R0 + kPairObj, lane);
      __syncwarp();
    }
    const int64_t un = u + rg.stride;
    const int64_t s0 = (t0 << 5) + lane;
    uint32_t g = p.k.gscal;
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[0], phase))) {
      if (lane == 0) report_timeout(p.k.err, &bars[0], phase);
      mbar_wait_bounded(&bars[1], phase);  // the other group's copies (bounded)
      break;
    }
    dp G[18];
    pair_hold(SG_, G, g);
    if (fx.ptr != nullptr) pair_grad<true, OX::adj, OY::adj>(fx, s0, mu, has1, G, SBY, g);
    else SBY.guard(g);
    fence_proxy_async_smem();
    __syncwarp();
    if (un < rg.end) pair_issue_adj<Tree>(lane, p, 2 * un, ntiles, mu, buf, bars, 0);
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[1], phase))) {
      if (lane == 0) report_timeout(p.k.err, &bars[1], phase);
      if (un < rg.end) mbar_wait_bounded(&bars[0], phase ^ 1);
      break;
    }
    if (fy.ptr != nullptr) pair_grad<false, OX::adj, OY::adj>(fy, s0, mu, has1, G, SBX, g);
    else SBX.guard(g);
    fence_proxy_async_smem();
    __syncwarp();
    if (un < rg.end) pair_issue_adj<Tree>(lane, p, 2 * un, ntiles, mu, buf, bars, 1);
    phase ^= 1;
    // the gradients overlap no input, so a unit with a site out of range is
    // rewritten in native FP64 after the pass
    if (__any_sync(0xffffffffu, guard_trips<Tree>(g))) {
      adj_site_f64<Tree>(p, s0, mu);
      if (has1) adj_site_f64<Tree>(p, s0 + 32, mu);
    }
    u = un;
  }
}

}  // namespace su3s
