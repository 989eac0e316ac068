// Device-side field access: addressing in the SoA / site-blocked layouts and
// loads/stores of whole site objects in each storage precision.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dev_math.cuh"
#include "kparams.h"

namespace su3s {

__device__ __forceinline__ int64_t elem_base(const FieldDesc& f, int64_t s, int mu) {
  return (s >> f.logB) * f.s_blk + (int64_t)mu * f.s_mu + (s & (int64_t)f.mask);
}

// Streaming 16-byte accesses (evict-first: every byte is touched once).
__device__ __forceinline__ uint4 ld16(const void* p) {
  uint4 v;
  asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void st16(void* p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint2 ld8(const void* p) {
  uint2 v;
  asm volatile("ld.global.cs.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ void st8(void* p, uint2 v) {
  asm volatile("st.global.cs.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(v.x), "r"(v.y) : "memory");
}

__device__ __forceinline__ double u2d(uint32_t lo, uint32_t hi) {
  return __hiloint2double((int)hi, (int)lo);
}

// --------------------------------------------------------------- storages
// Each storage moves one complex component of VPS consecutive sites with one
// vector access.  Values are produced in the arithmetic of Math (FP64 storage:
// Math::from_bits; an object is complete after Math::normalize_obj).

template <int PREC>
struct Store;

// FP64: 16 bytes = one complex of one site.
template <>
struct Store<P_F64> {
  static constexpr int VPS = 1;
  static constexpr int kElemBytes = 16;
  template <class M>
  __device__ static __forceinline__ void load(const void* base, int64_t e, typename M::R* re,
                                              typename M::R* im) {
    uint4 v = ld16((const char*)base + e * 16);
    split_complex<M>(v, re[0], im[0]);
  }
  // from accumulators
  template <class M>
  __device__ static __forceinline__ void store_acc(void* base, int64_t e, const typename M::A* re,
                                                   const typename M::A* im) {
    double r, i;
    complex_to_f64<M>(re[0], im[0], r, i);
    st16((char*)base + e * 16, make_uint4((uint32_t)__double2loint(r), (uint32_t)__double2hiint(r),
                                          (uint32_t)__double2loint(i), (uint32_t)__double2hiint(i)));
  }
};

// Reduced precisions: two sites per access.
template <>
struct Store<P_F32> {
  static constexpr int VPS = 2;
  static constexpr int kElemBytes = 8;
  template <class M>
  __device__ static __forceinline__ void load(const void* base, int64_t e, float* re, float* im) {
    uint4 v = ld16((const char*)base + e * 8);
    re[0] = __uint_as_float(v.x);
    im[0] = __uint_as_float(v.y);
    re[1] = __uint_as_float(v.z);
    im[1] = __uint_as_float(v.w);
  }
  template <class M>
  __device__ static __forceinline__ void store_acc(void* base, int64_t e, const float* re,
                                                   const float* im) {
    st16((char*)base + e * 8, make_uint4(__float_as_uint(re[0]), __float_as_uint(im[0]),
                                         __float_as_uint(re[1]), __float_as_uint(im[1])));
  }
};

template <>
struct Store<P_BF16> {
  static constexpr int VPS = 2;
  static constexpr int kElemBytes = 4;
  template <class M>
  __device__ static __forceinline__ void load(const void* base, int64_t e, float* re, float* im) {
    uint2 v = ld8((const char*)base + e * 4);
    re[0] = __uint_as_float(v.x << 16);
    im[0] = __uint_as_float(v.x & 0xFFFF0000u);
    re[1] = __uint_as_float(v.y << 16);
    im[1] = __uint_as_float(v.y & 0xFFFF0000u);
  }
  template <class M>
  __device__ static __forceinline__ void store_acc(void* base, int64_t e, const float* re,
                                                   const float* im) {
    __nv_bfloat162 p0 = __floats2bfloat162_rn(re[0], im[0]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(re[1], im[1]);
    st8((char*)base + e * 4,
        make_uint2(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1)));
  }
};

template <>
struct Store<P_F16> {
  static constexpr int VPS = 2;
  static constexpr int kElemBytes = 4;
  template <class M>
  __device__ static __forceinline__ void load(const void* base, int64_t e, float* re, float* im) {
    uint2 v = ld8((const char*)base + e * 4);
    __half2 h0 = *reinterpret_cast<__half2*>(&v.x);
    __half2 h1 = *reinterpret_cast<__half2*>(&v.y);
    float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    re[0] = f0.x;
    im[0] = f0.y;
    re[1] = f1.x;
    im[1] = f1.y;
  }
  template <class M>
  __device__ static __forceinline__ void store_acc(void* base, int64_t e, const float* re,
                                                   const float* im) {
    __half2 p0 = __floats2half2_rn(re[0], im[0]);
    __half2 p1 = __floats2half2_rn(re[1], im[1]);
    st8((char*)base + e * 4,
        make_uint2(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1)));
  }
};

// Storage of C12 matrices uses the complex element of the base precision.
template <int PREC>
struct BaseStore {
  using type = Store<PREC>;
};
template <>
struct BaseStore<P_F64_C12> {
  using type = Store<P_F64>;
};
template <>
struct BaseStore<P_F32_C12> {
  using type = Store<P_F32>;
};

// Real fields (FP64 only): one double per site object, VPS = 1.  Values
// come back as Math::from_bits; the caller normalises the object.
struct StoreReal {
  template <class M>
  __device__ static __forceinline__ typename M::R load(const void* base, int64_t e) {
    uint2 v = ld8((const char*)base + e * 8);
    return M::from_bits(v.x, v.y);
  }
  template <class M>
  __device__ static __forceinline__ void store_acc(void* base, int64_t e, const typename M::A& a) {
    double r = M::to_f64(a);
    st8((char*)base + e * 8, make_uint2((uint32_t)__double2loint(r), (uint32_t)__double2hiint(r)));
  }
};

}  // namespace su3s
