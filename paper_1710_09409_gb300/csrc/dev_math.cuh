// Arithmetic policies for site-local complex 3x3 algebra on sm_103a.
//
//   MathF64  native IEEE FP64 with fused multiply-add.  On the GB300 the FP64
//            pipe retires about two DFMA per clock per SM, so a 3x3 complex
//            product (108 DFMA) caps near 5 G sites/s, far below HBM speed.
//   MathDF   FP64-accurate arithmetic from FP32 and integer instructions only
//            (no FP64 instruction, not even a conversion, all of which run on
//            the narrow FP64 pipe):
//              * an FP64 input x is split by bit operations into a pair of
//                FP32 values xh + xl with |x - xh - xl| <= 2^-48 |x|
//                (xh = x truncated to 24 significant bits, xl = the remaining
//                29 bits rounded to 24 by an integer-to-float conversion);
//              * a sum of products sum_t x_t*y_t keeps a running FP32 sum S of
//                the leading products xh*yh and an FP32 tail `lo`; each new
//                leading product enters S through Knuth's TwoSum, whose error
//                term is taken with an FMA against the exact product so the
//                product's own rounding error folds in; that error and the
//                cross terms xh*yl + xl*yh are gathered per term and enter the
//                tail with one rounding (Dekker/Knuth error-free
//                transformations, Ogita-Rump-Oishi style dot product);
//              * the result S + lo is rounded toward zero into one FP32 value
//                plus a same-signed remainder, and the FP64 bit pattern is
//                assembled with integer operations: the leading value gives
//                sign, exponent and the top 23 fraction bits, the remainder
//                scaled to units of the last place gives the low 29 bits.
//            Error per output ~2^-46 * sum_t |x_t y_t| + 2^-52 |z|.  Needs all
//            magnitudes below 2^126; magnitudes below 2^-126 may be flushed.
//            3x3 complex products run the real and imaginary accumulations of
//            an output in the two lanes of packed FP32 instructions (same
//            operations per lane, fewer issued instructions); MathDFScalar is
//            the scalar-issue form for kernels short of registers.
//   MathFX   FP64-accurate arithmetic on the integer multiply-add units
//            (shared-exponent fixed point):
//              * the reals of one site object (a matrix, a vector, a real)
//                share one exponent E, that of the object's largest element;
//                each real becomes a signed integer m = x * 2^(1075-E) with
//                |m| < 2^53 (the 53-bit significand shifted right by the
//                element's exponent gap, truncated; negative values take the
//                one's complement), held as m = h*2^25 + l;
//              * a product term x*y is h_x*h_y (one 32x32->64-bit multiply-add)
//                plus the cross terms h_x*l_y + l_x*h_y, whose high 32 bits
//                are accumulated (two multiply-high-adds); l_x*l_y, below the
//                accumulator's unit, is dropped.  Every term of one product
//                shares the scale E_x + E_y, so a 3x3 complex product is 108
//                exact integer multiply-adds into 64-bit accumulators;
//              * sums of products with different scales are aligned by
//                arithmetic shifts; an intermediate object is renormalised to
//                a shared exponent; the result is converted with one
//                int64 -> FP64 conversion and an exponent adjustment.
//            Error per output <= ~2^-47 * 6 * max|x| * max|y| over the two
//            operand objects (absolute, relative to the objects' largest
//            elements).  Objects whose largest magnitude is below 2^-958 are
//            flushed to zero; results must stay below 2^960 in magnitude.
//   MathF32  FP32 arithmetic for FP32/BF16/FP16 storage (FP32 accumulation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace su3s {

// ----------------------------------------------------------------- helpers
struct df {
  float h, l;
};

// FP64 bit pattern (lo32, hi32) -> (xh, xl).  No FP64 instruction.
//
// Integer part of the split: hb = the bits of xh, m = the low 29 mantissa
// bits as an FP32 value (xl = m * 2^(E-52), with E the exponent of xh).
__device__ __forceinline__ void df_split_head(uint32_t lo32, uint32_t hi32, uint32_t& hb, float& m) {
  // rebias 1023 -> 127; exponents below 2^-126 collapse to 0 (fused add + max)
  const uint32_t w = (uint32_t)__viaddmax_s32((int)(hi32 & 0x7FFFFFFFu), -0x38000000, 0);
  const uint32_t t = __funnelshift_l(lo32, w, 3);  // exponent + top 23 fraction bits
  hb = t | (hi32 & 0x80000000u);
  m = __uint2float_rn(lo32 & 0x1FFFFFFFu);         // low 29 bits
}

// The split itself.
__device__ __forceinline__ df df_split_bits(uint32_t lo32, uint32_t hi32) {
  uint32_t hb;
  float m;
  df_split_head(lo32, hi32, hb, m);
  float pw = __fmul_rn(__uint_as_float(hb & 0xFF800000u), 0x1p-52f);    // +-2^(E-52)
  return df{__uint_as_float(hb), __fmul_rn(m, pw)};
}

// The FP64 bit pattern of s + e, s a sum rounded toward zero and e its exact
// remainder (same sign as s, below one unit of s's last place).
__device__ __forceinline__ double df_assemble(float s, float e) {
  uint32_t fs = __float_as_uint(s);
  uint32_t fa = fs & 0x7FFFFFFFu;
  uint32_t sg = fs & 0x80000000u;
  float pw = __uint_as_float((306u << 23) - (fa & 0x7F800000u));        // 2^(52 - E_s)
  uint32_t low29 = min(__float2uint_rz(__fmul_rn(fabsf(e), pw)), 0x1FFFFFFFu);
  uint32_t hiw = ((fa >> 3) + 0x38000000u) | sg;
  hiw = fa ? hiw : sg;
  uint32_t low = fs * 0x20000000u + low29;  // (fs << 29) | low29; both zero when s == 0
  return __hiloint2double((int)hiw, (int)low);
}

// (S, lo) with |lo| << |S| (not necessarily normalised) -> FP64.
__device__ __forceinline__ double df_to_double(float S, float lo) {
  float s = __fadd_rz(S, lo);          // toward zero: the remainder shares s's sign
  float z = __fsub_rn(s, S);
  float e = __fsub_rn(lo, z);
  return df_assemble(s, e);
}

// Normalise (S, lo) into a pair usable as an operand: Fast2Sum.
__device__ __forceinline__ df df_norm(float S, float lo) {
  float h = __fadd_rn(S, lo);
  float l = __fsub_rn(lo, __fsub_rn(h, S));
  return df{h, l};
}

// ------------------------------------------------------------ range guard
// The FP64-accurate arithmetics hold FP64 values in narrower formats: MathDF
// in FP32 pairs, whose exponent range ends at 2^128 (an FP64 input at or above
// it does not split; products and sums of large inputs overflow the leading
// parts), MathFX in integers scaled by per-object exponents (bounded results).
// Neither represents Inf or NaN.  Kernels that evaluate in them therefore
// keep, per site, the largest magnitude among the site's FP64 inputs (leaves,
// dL/dZ, real factors) as the maximum of the inputs' high words with the sign
// cleared: non-negative FP64 values order as their bit patterns, and Inf and
// NaN come after every finite value.  A site whose maximum reaches its tree's
// bound 2^t(d) is evaluated again in native FP64 from its inputs in global
// memory, before anything of it is stored, so every input gets the IEEE
// result (NaN, Inf, values beyond FP32 range).  d is the tree's degree (the
// most factors, leaves and real factors, in one product term); with
// t(d) = floor((120 - 3 (d - 1)) / d) every term, partial sum and TwoSum
// intermediate of a site in range stays below 2^127 (a 3x3 complex product
// term sums at most 6 |x||y| per real; a degree-3 term at most 36 of them).
// Magnitudes below 2^-126 are not guarded: MathDF flushes them, an absolute
// error below 2^-126 times the other factors' magnitudes.
__host__ __device__ constexpr uint32_t guard_hi(int degree) {
  return (uint32_t)(1023 + (120 - 3 * (degree - 1)) / degree) << 20;
}

// running maximum of two inputs' high words (sign bits cleared)
__device__ __forceinline__ uint32_t guard_max(uint32_t g, uint32_t hi_a, uint32_t hi_b) {
  return __vimax3_u32(g, hi_a & 0x7FFFFFFFu, hi_b & 0x7FFFFFFFu);
}

// maximum of N per-element guard words by a pairwise tree (depth log2 N, so
// it completes as soon as the object is read)
template <int N>
__device__ __forceinline__ uint32_t guard_reduce(uint32_t* g) {
#pragma unroll
  for (int w = 1; w < N; w *= 2)
#pragma unroll
    for (int i = 0; i + w < N; i += 2 * w) g[i] = max(g[i], g[i + w]);
  return g[0];
}

// ------------------------------------------------------------- MathF64
struct MathF64 {
  using R = double;   // one real component
  using A = double;   // accumulator
  static constexpr bool kScaled = false;  // every term shares one scale
  static constexpr bool kPaired = false;  // no packed (re, im) products
  static constexpr bool kGuard = false;   // IEEE semantics for every input
  __device__ static __forceinline__ R from_bits(uint32_t lo, uint32_t hi) {
    return __hiloint2double((int)hi, (int)lo);
  }
  template <int W>
  __device__ static __forceinline__ void normalize_obj(R*) {}
  __device__ static __forceinline__ double to_f64(const A& a) { return a; }
  __device__ static __forceinline__ R finish(const A& a) { return a; }
  __device__ static __forceinline__ A to_acc(const R& x) { return x; }
  __device__ static __forceinline__ A zero() { return 0.0; }
  __device__ static __forceinline__ R neg(const R& x) { return -x; }
  __device__ static __forceinline__ R scalar(double s, float, float) { return s; }
  // a (+)= sg * x * y ; FIRST: a = sg * x * y
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void fma(A& a, const R& x, const R& y) {
    if (FIRST) a = (SG > 0) ? __dmul_rn(x, y) : __dmul_rn(-x, y);
    else a = (SG > 0) ? __fma_rn(x, y, a) : __fma_rn(-x, y, a);
  }
  // a (+)= sg * x
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void add(A& a, const R& x) {
    if (FIRST) a = (SG > 0) ? x : -x;
    else a = (SG > 0) ? __dadd_rn(a, x) : __dsub_rn(a, x);
  }
  // a += sg * b for two accumulators
  template <int SG>
  __device__ static __forceinline__ void combine(A& a, const A& b) {
    a = (SG > 0) ? __dadd_rn(a, b) : __dsub_rn(a, b);
  }
};

// -------------------------------------------------------------- MathDF
struct DAcc {
  float S, lo;
};

struct MathDF {
  using R = df;
  using A = DAcc;
  static constexpr bool kScaled = false;
  static constexpr bool kPaired = true;   // complex products in packed (re, im) lanes
  static constexpr bool kGuard = true;    // FP32 exponent range: sites are range-checked
  static constexpr bool kPackSplit = true;  // complex inputs split, outputs converted, in pairs
  __device__ static __forceinline__ R from_bits(uint32_t lo, uint32_t hi) {
    return df_split_bits(lo, hi);
  }
  template <int W>
  __device__ static __forceinline__ void normalize_obj(R*) {}
  __device__ static __forceinline__ double to_f64(const A& a) { return df_to_double(a.S, a.lo); }
  __device__ static __forceinline__ R finish(const A& a) { return df_norm(a.S, a.lo); }
  __device__ static __forceinline__ A to_acc(const R& x) { return DAcc{x.h, x.l}; }
  __device__ static __forceinline__ A zero() { return DAcc{0.0f, 0.0f}; }
  __device__ static __forceinline__ R neg(const R& x) { return df{-x.h, -x.l}; }
  __device__ static __forceinline__ R scalar(double, float sh, float sl) { return df{sh, sl}; }

  template <bool FIRST, int SG>
  __device__ static __forceinline__ void fma(A& a, const R& x0, const R& y) {
    const float xh = SG > 0 ? x0.h : -x0.h;
    const float xl = SG > 0 ? x0.l : -x0.l;
    // The leading product is formed as xh*yh + (+0): the rounded product,
    // except that an exact -0 comes out as +0 (TwoSum below is exact for any
    // float p).  Its packed form, fma.rn.f32x2 with a +0 addend, is not a
    // plain multiply, which the compiler would merge into the add after it.
    const float p = __fmaf_rn(xh, y.h, 0.0f);
    if (FIRST) {
      float q = __fmaf_rn(xh, y.h, -p);       // exact error of the leading product
      q = __fmaf_rn(xh, y.l, q);
      q = __fmaf_rn(xl, y.h, q);
      a.S = p;
      a.lo = q;
    } else {
      const float s = __fadd_rn(a.S, p);       // TwoSum(S, xh*yh)
      const float bp = __fsub_rn(s, a.S);
      const float ap = __fsub_rn(s, bp);
      const float db = __fmaf_rn(xh, y.h, -bp);  // exact product minus bp, one rounding
      const float da = __fsub_rn(a.S, ap);
      // this term's small parts (sum error, cross terms) are gathered first and
      // enter the running tail with a single rounding
      float t = __fadd_rn(da, db);
      t = __fmaf_rn(xl, y.h, t);
      t = __fmaf_rn(xh, y.l, t);
      a.S = s;
      a.lo = __fadd_rn(a.lo, t);
    }
  }

  // a += sg * b for two accumulators: TwoSum of the leading parts, tails added
  template <int SG>
  __device__ static __forceinline__ void combine(A& a, const A& b0) {
    const float bS = SG > 0 ? b0.S : -b0.S;
    const float bl = SG > 0 ? b0.lo : -b0.lo;
    const float s = __fadd_rn(a.S, bS);
    const float bp = __fsub_rn(s, a.S);
    const float ap = __fsub_rn(s, bp);
    const float db = __fsub_rn(bS, bp);
    const float da = __fsub_rn(a.S, ap);
    float t = __fadd_rn(da, db);
    t = __fadd_rn(t, bl);
    a.S = s;
    a.lo = __fadd_rn(a.lo, t);
  }

  template <bool FIRST, int SG>
  __device__ static __forceinline__ void add(A& a, const R& x0) {
    const float xh = SG > 0 ? x0.h : -x0.h;
    const float xl = SG > 0 ? x0.l : -x0.l;
    if (FIRST) {
      a.S = xh;
      a.lo = xl;
    } else {
      const float s = __fadd_rn(a.S, xh);
      const float bp = __fsub_rn(s, a.S);
      const float ap = __fsub_rn(s, bp);
      const float db = __fsub_rn(xh, bp);
      const float da = __fsub_rn(a.S, ap);
      float t = __fadd_rn(da, db);
      t = __fadd_rn(t, xl);
      a.S = s;
      a.lo = __fadd_rn(a.lo, t);
    }
  }
};

// The same arithmetic issued as scalar instructions only, for kernels whose
// register budget has no room for the packed operand pairs (the reverse mode
// of multi-product trees, the hopping term on matrices, the interpreter):
// there the extra registers of the pairs cost more than the packed
// instructions save.  Results are identical to MathDF's.
struct MathDFScalar : MathDF {
  static constexpr bool kPaired = false;
};

// The same arithmetic with every FP64 input split and every output converted
// one real at a time (MathDF packs the two reals of a complex element: the
// same values).  Measured faster for the Wilson term, whose schedule lost more
// to the packed operations' register pairs than the packing saved (48^4:
// 1,923 against 1,887 GB/s).
struct MathDFUnpacked : MathDF {
  static constexpr bool kPackSplit = false;
};

// --------------------------------------------- MathDF, packed (re, im) lanes
// The real and imaginary parts of one complex output advance together in the
// two lanes of the packed FP32 instructions of sm_100 and later (two FP32
// operations per issued instruction).  Each lane performs exactly the
// operations of MathDF::fma / MathDF::combine in the same order, so the packed
// path gives the same values as the scalar one.  Adds, subtracts and FMAs are
// packed (PTX with an explicit round-to-nearest-even modifier), and so is the
// leading product, as an FMA with a +0 addend.  With CUDA 13.0 on sm_103a a
// packed multiply whose result fed a packed add was merged with it into one
// FMA, which loses TwoSum's exact error term (the 3x3 product came out with
// FP32 accuracy, ~1e-8), and so was an FMA with a -0 addend (exactly a
// multiply); an FMA with a +0 addend differs from a multiply for a -0 product
// and is kept apart.  -bp is formed as S - s, the exact negation of s - S
// under round-to-nearest-even.
struct DAcc2 {
  float2 S, lo;  // .x = real part's accumulator, .y = imaginary part's
};
struct df2 {
  float2 h, l;   // lane-wise leading and trailing parts
};

// lane-wise leading product x.h * y.h + (+0) (MathDF::fma's p)
__device__ __forceinline__ float2 f2_mul_lead(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, 0;\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ DAcc2 dacc2_get(const DAcc& re, const DAcc& im) {
  return DAcc2{make_float2(re.S, im.S), make_float2(re.lo, im.lo)};
}
__device__ __forceinline__ void dacc2_put(DAcc& re, DAcc& im, const DAcc2& a) {
  re.S = a.S.x;
  im.S = a.S.y;
  re.lo = a.lo.x;
  im.lo = a.lo.y;
}

// a = x * y lane-wise (MathDF::fma with FIRST)
__device__ __forceinline__ void df2_first(DAcc2& a, const df2& x, const df2& y) {
  const float2 p = f2_mul_lead(x.h, y.h);
  const float2 np = make_float2(-p.x, -p.y);
  float2 q = f2_fma(x.h, y.h, np);            // exact error of the leading product
  q = f2_fma(x.h, y.l, q);
  q = f2_fma(x.l, y.h, q);
  a.S = p;
  a.lo = q;
}

// a += x * y lane-wise (MathDF::fma without FIRST)
__device__ __forceinline__ void df2_fma(DAcc2& a, const df2& x, const df2& y) {
  const float2 p = f2_mul_lead(x.h, y.h);
  const float2 s = f2_add(a.S, p);            // TwoSum(S, xh*yh)
  const float2 nbp = f2_sub(a.S, s);          // -bp
  const float2 ap = f2_add(s, nbp);           // s - bp
  const float2 db = f2_fma(x.h, y.h, nbp);    // exact product minus bp, one rounding
  const float2 da = f2_sub(a.S, ap);
  float2 t = f2_add(da, db);
  t = f2_fma(x.l, y.h, t);
  t = f2_fma(x.h, y.l, t);
  a.S = s;
  a.lo = f2_add(a.lo, t);
}

// a += SG * b lane-wise (MathDF::combine)
template <int SG>
__device__ __forceinline__ void df2_combine(DAcc2& a, const DAcc2& b) {
  const float2 s = SG > 0 ? f2_add(a.S, b.S) : f2_sub(a.S, b.S);
  const float2 nbp = f2_sub(a.S, s);          // -bp
  const float2 ap = f2_add(s, nbp);           // s - bp
  const float2 db = SG > 0 ? f2_add(b.S, nbp) : f2_sub(nbp, b.S);  // sg*bS - bp
  const float2 da = f2_sub(a.S, ap);
  float2 t = f2_add(da, db);
  t = SG > 0 ? f2_add(t, b.lo) : f2_sub(t, b.lo);
  a.S = s;
  a.lo = f2_add(a.lo, t);
}

// -------------------------------------------------------------- MathFX
// One real of an object: value (h * 2^25 + l * 2^-6) * 2^(e - 1075), with
// |h| <= 2^28, |l| < 2^31 and l a multiple of 64 (the low 25 bits of m,
// pre-shifted for the multiply-high of the cross terms).  e is the object's
// shared exponent; before normalize_obj, (h, l) hold the raw FP64 bits.
struct fxr {
  int h, l, e;
};
// Accumulator: value (hh + 2 * cr) * 2^(e - 2100).
struct FAcc {
  long long hh;
  int cr, e;
};

constexpr int kFxEmin = 64;         // biased exponent floor of an object
constexpr int kFxZeroE = -(1 << 20);  // scale of an empty accumulator

// Shifts with PTX semantics: amounts beyond 63 give 0 (logical) or the sign
// (arithmetic).
__device__ __forceinline__ uint64_t fx_shr(uint64_t x, uint32_t s) {
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}
__device__ __forceinline__ long long fx_sar(long long x, uint32_t s) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}
__device__ __forceinline__ long long fx_total(const FAcc& a) {
  return a.hh + ((long long)a.cr << 1);
}

struct MathFX {
  using R = fxr;
  using A = FAcc;
  static constexpr bool kScaled = true;  // terms of different objects differ in scale
  static constexpr bool kPaired = false;
  static constexpr bool kGuard = true;   // finite inputs of bounded scale: range-checked

  __device__ static __forceinline__ R from_bits(uint32_t lo, uint32_t hi) {
    return fxr{(int)hi, (int)lo, 0};
  }
  // Raw FP64 bits of W reals -> shared-exponent fixed point.
  template <int W>
  __device__ static __forceinline__ void normalize_obj(R* x) {
    // largest magnitude by a pairwise tree (depth log2 W, not a W-long chain)
    uint32_t m[W];
#pragma unroll
    for (int i = 0; i < W; ++i) m[i] = (uint32_t)x[i].h & 0x7FFFFFFFu;
#pragma unroll
    for (int w = 1; w < W; w *= 2)
#pragma unroll
      for (int i = 0; i + w < W; i += 2 * w) m[i] = max(m[i], m[i + w]);
    const uint32_t amax = m[0];
    const int E = max((int)(amax >> 20), kFxEmin);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint32_t hi = (uint32_t)x[i].h, lo = (uint32_t)x[i].l;
      const uint32_t ah = hi & 0x7FFFFFFFu;
      // zero and subnormal elements have exponent 0: their gap is >= 64
      const uint32_t d = (uint32_t)(E - (int)(ah >> 20));
      const uint64_t M = ((uint64_t)((ah & 0xFFFFFu) | 0x100000u) << 32) | lo;
      const uint64_t m = fx_shr(M, d);
      const uint32_t sg = (uint32_t)((int)hi >> 31);
      x[i].h = (int)((uint32_t)(m >> 25) ^ sg);
      x[i].l = (int)((((uint32_t)m << 6) ^ sg) & 0x7FFFFFC0u);
      x[i].e = E;
    }
  }
  // W accumulators (scales may differ) -> one object with a shared exponent.
  template <int W>
  __device__ static __forceinline__ void finish_obj(R* out, const A* a) {
    // largest scale and the OR of the magnitudes by pairwise trees
    int es[W];
#pragma unroll
    for (int i = 0; i < W; ++i) es[i] = a[i].e;
#pragma unroll
    for (int w = 1; w < W; w *= 2)
#pragma unroll
      for (int i = 0; i + w < W; i += 2 * w) es[i] = max(es[i], es[i + w]);
    const int e = es[0];
    long long T[W];
    uint64_t ov[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      T[i] = fx_sar(fx_total(a[i]), (uint32_t)(e - a[i].e));
      ov[i] = (uint64_t)(T[i] ^ (T[i] >> 63));
    }
#pragma unroll
    for (int w = 1; w < W; w *= 2)
#pragma unroll
      for (int i = 0; i + w < W; i += 2 * w) ov[i] |= ov[i + w];
    const uint64_t orv = ov[0];
    const int sh = max(64 - __clzll((long long)orv) - 53, 0);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const long long m = fx_sar(T[i], (uint32_t)sh);
      out[i].h = (int)(m >> 25);
      out[i].l = (int)(((uint32_t)m << 6) & 0x7FFFFFC0u);
      out[i].e = e + sh - 1025;
    }
  }
  // Result: T = hh + 2 cr converted once (round to nearest even), then the
  // exponent field moved by the accumulator's scale.  Supported range: results
  // below 2^960 in magnitude; results below 2^-1022 come out as subnormals of
  // unspecified significand (absolute error below 2^-1022).
  __device__ static __forceinline__ double to_f64(const A& a) {
    const double d = __ll2double_rn(fx_total(a));
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const int ah = (int)(hi & 0x7FFFFFFFu);
    // d == 0 or its biased exponent is in [1023, 1085] (|T| < 2^62): with the
    // adjustment clamped to [-1100, 960] the new exponent stays below 2047
    const int k = min(max(a.e - 2100, -1100), 960) * (1 << 20);
    const int nh = max(ah + k * min(ah, 1), 0);
    return __hiloint2double((int)((uint32_t)nh | (hi & 0x80000000u)), __double2loint(d));
  }
  __device__ static __forceinline__ R finish(const A& a) {
    R r;
    finish_obj<1>(&r, &a);
    return r;
  }
  __device__ static __forceinline__ A to_acc(const R& x) {
    return FAcc{(long long)x.h * (1LL << 25) + (long long)(x.l >> 6), 0, x.e + 1025};
  }
  __device__ static __forceinline__ A zero() { return FAcc{0, 0, kFxZeroE}; }
  __device__ static __forceinline__ R neg(const R& x) { return fxr{-x.h, -x.l, x.e}; }
  __device__ static __forceinline__ R scalar(double s, float, float) {
    R r = from_bits((uint32_t)__double2loint(s), (uint32_t)__double2hiint(s));
    normalize_obj<1>(&r);
    return r;
  }

  // a (+)= SG * x * y.  Not FIRST: a's scale must be x.e + y.e (terms of one
  // product); terms of other scales go through combine.
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void fma(A& a, const R& x, const R& y) {
    const int xh = SG > 0 ? x.h : -x.h;
    const int xl = SG > 0 ? x.l : -x.l;
    if (FIRST) {
      a.hh = (long long)xh * y.h;
      a.cr = __mulhi(xh, y.l) + __mulhi(xl, y.h);
      a.e = x.e + y.e;
    } else {
      a.hh += (long long)xh * y.h;
      a.cr += __mulhi(xh, y.l);
      a.cr += __mulhi(xl, y.h);
    }
  }
  // fold the cross-term sum into the 64-bit part (frees a register per
  // accumulator that is no longer multiplied into)
  __device__ static __forceinline__ void compact(A& a) {
    a.hh = fx_total(a);
    a.cr = 0;
  }
  // a += SG * b at the larger of the two scales
  template <int SG>
  __device__ static __forceinline__ void combine(A& a, const A& b) {
    const int e = max(a.e, b.e);
    const long long ta = fx_sar(fx_total(a), (uint32_t)(e - a.e));
    const long long tb = fx_sar(fx_total(b), (uint32_t)(e - b.e));
    a.hh = SG > 0 ? ta + tb : ta - tb;
    a.cr = 0;
    a.e = e;
  }
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void add(A& a, const R& x) {
    const A t = to_acc(SG > 0 ? x : neg(x));
    if (FIRST) a = t;
    else combine<1>(a, t);
  }
};

// ------------------------------------------------------------- MathF32
struct MathF32 {
  using R = float;
  using A = float;
  static constexpr bool kScaled = false;
  static constexpr bool kPaired = false;
  static constexpr bool kGuard = false;
  __device__ static __forceinline__ R finish(const A& a) { return a; }
  __device__ static __forceinline__ A to_acc(const R& x) { return x; }
  __device__ static __forceinline__ A zero() { return 0.0f; }
  __device__ static __forceinline__ R neg(const R& x) { return -x; }
  __device__ static __forceinline__ R scalar(double, float sh, float) { return sh; }
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void fma(A& a, const R& x, const R& y) {
    if (FIRST) a = (SG > 0) ? __fmul_rn(x, y) : __fmul_rn(-x, y);
    else a = (SG > 0) ? __fmaf_rn(x, y, a) : __fmaf_rn(-x, y, a);
  }
  template <bool FIRST, int SG>
  __device__ static __forceinline__ void add(A& a, const R& x) {
    if (FIRST) a = (SG > 0) ? x : -x;
    else a = (SG > 0) ? __fadd_rn(a, x) : __fsub_rn(a, x);
  }
  template <int SG>
  __device__ static __forceinline__ void combine(A& a, const A& b) {
    a = (SG > 0) ? __fadd_rn(a, b) : __fsub_rn(a, b);
  }
};

// ------------------------------------------ complex elements, two reals
// Packed product, used only where it feeds another product: a packed
// multiply feeding a packed add is not kept apart from it (see f2_mul_lead).
__device__ __forceinline__ float2 f2_mul_packed(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_add_rz(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rz.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// df_split_bits of two FP64 values (lane 0: (lo0, hi0), lane 1: (lo1, hi1)),
// its two FP32 multiplies packed.
__device__ __forceinline__ df2 df2_split(uint32_t lo0, uint32_t hi0, uint32_t lo1, uint32_t hi1) {
  uint32_t hb0, hb1;
  float m0, m1;
  df_split_head(lo0, hi0, hb0, m0);
  df_split_head(lo1, hi1, hb1, m1);
  const float2 pw = f2_mul_packed(make_float2(__uint_as_float(hb0 & 0xFF800000u),
                                              __uint_as_float(hb1 & 0xFF800000u)),
                                  make_float2(0x1p-52f, 0x1p-52f));  // +-2^(E-52)
  return df2{make_float2(__uint_as_float(hb0), __uint_as_float(hb1)),
             f2_mul_packed(make_float2(m0, m1), pw)};
}

// df_to_double of two accumulators (lanes of a DAcc2), its FP32 operations packed.
__device__ __forceinline__ void df2_to_double(const DAcc2& a, double& d0, double& d1) {
  const float2 s = f2_add_rz(a.S, a.lo);  // toward zero: the remainder shares s's sign
  const float2 z = f2_sub(s, a.S);
  const float2 e = f2_sub(a.lo, z);
  d0 = df_assemble(s.x, e.x);
  d1 = df_assemble(s.y, e.y);
}

// Whether M splits and converts complex elements in packed pairs.
template <class M>
__host__ __device__ constexpr bool pack_split() {
  if constexpr (std::is_base_of<MathDF, M>::value) return M::kPackSplit;
  else return false;
}

// One complex element (16 bytes: re lo, re hi, im lo, im hi) into the
// arithmetic's two reals.  The pair arithmetic splits both at once with its
// multiplies packed over (re, im); each lane repeats df_split_bits, so the
// values are those of from_bits.
template <class M>
__device__ __forceinline__ void split_complex(uint4 v, typename M::R& re, typename M::R& im) {
  if constexpr (pack_split<M>()) {
    const df2 p = df2_split(v.x, v.y, v.z, v.w);
    re = df{p.h.x, p.l.x};
    im = df{p.h.y, p.l.y};
  } else {
    re = M::from_bits(v.x, v.y);
    im = M::from_bits(v.z, v.w);
  }
}

// The FP64 values of a complex output's two accumulators (packed for the pair
// arithmetic, with to_f64's values).
template <class M>
__device__ __forceinline__ void complex_to_f64(const typename M::A& re, const typename M::A& im,
                                               double& r, double& i) {
  if constexpr (pack_split<M>()) {
    df2_to_double(DAcc2{make_float2(re.S, im.S), make_float2(re.lo, im.lo)}, r, i);
  } else {
    r = M::to_f64(re);
    i = M::to_f64(im);
  }
}

}  // namespace su3s
