// Element-wise conversion between FP64 values and stored complex elements of
// each precision (round to nearest even on narrowing, exact on widening).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kparams.h"

namespace su3s {

__device__ __forceinline__ int64_t fbase(const FieldDesc& d, int64_t s, int mu) {
  return (s >> d.logB) * d.s_blk + (int64_t)mu * d.s_mu + (s & (int64_t)d.mask);
}

template <int PREC>
__device__ __forceinline__ void put_complex(void* base, int64_t e, double re, double im) {
  if constexpr (PREC == P_F64 || PREC == P_F64_C12) {
    reinterpret_cast<double2*>(base)[e] = make_double2(re, im);
  } else if constexpr (PREC == P_F32 || PREC == P_F32_C12) {
    reinterpret_cast<float2*>(base)[e] = make_float2(__double2float_rn(re), __double2float_rn(im));
  } else if constexpr (PREC == P_BF16) {
    __nv_bfloat162 v;
    v.x = __double2bfloat16(re);
    v.y = __double2bfloat16(im);
    reinterpret_cast<__nv_bfloat162*>(base)[e] = v;
  } else {
    __half2 v;
    v.x = __double2half(re);
    v.y = __double2half(im);
    reinterpret_cast<__half2*>(base)[e] = v;
  }
}

template <int PREC>
__device__ __forceinline__ double2 get_complex(const void* base, int64_t e) {
  if constexpr (PREC == P_F64 || PREC == P_F64_C12) {
    return reinterpret_cast<const double2*>(base)[e];
  } else if constexpr (PREC == P_F32 || PREC == P_F32_C12) {
    float2 v = reinterpret_cast<const float2*>(base)[e];
    return make_double2((double)v.x, (double)v.y);
  } else if constexpr (PREC == P_BF16) {
    __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162*>(base)[e];
    return make_double2((double)__bfloat162float(v.x), (double)__bfloat162float(v.y));
  } else {
    __half2 v = reinterpret_cast<const __half2*>(base)[e];
    return make_double2((double)__half2float(v.x), (double)__half2float(v.y));
  }
}

}  // namespace su3s
