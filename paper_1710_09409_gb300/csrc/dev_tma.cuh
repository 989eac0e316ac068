// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with
// mbarrier completion, used to stage the next tile of a warp's sites while
// the warp computes the current one.
//
// Every wait is bounded: after kTmaSpinLimit polls the waiting warp records
// an error code in the library's device error word (KParams::err), waits once
// more (again bounded) for its own copies in flight, and leaves its loop.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace su3s {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t smem_u32_base(const void* p) { return smem_u32(p); }

// A poll that finds the phase incomplete suspends the thread for ~7,800 SM
// cycles (measured with su3s_selftest_bounded_wait on GB300: ~3.8 us), so
// 2^18 polls give up after about one second, a million times the latency of a
// tile's copies.
constexpr uint32_t kTmaSpinLimit = 1u << 18;
constexpr int kErrTmaTimeout = 1;
constexpr int kErrSmemAlign = 2;   // dynamic shared memory not 128-byte aligned: nothing staged

// Tensor copies need 128-byte aligned shared-memory destinations; a kernel
// whose dynamic shared memory is not aligned records the fact and stages
// nothing (all its warps return before any copy).
__device__ __forceinline__ bool smem_aligned(const void* smem, int* err) {
  if ((smem_u32_base(smem) & 127u) == 0) return true;
  if (err && threadIdx.x == 0) atomicExch(err, kErrSmemAlign);
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` in bytes.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tensor copy global -> shared of the map's box at column x, row y,
// completion counted on `bar` in bytes.  dst 128-byte aligned; x times the
// element size a multiple of 16 bytes; the map lives in kernel parameter space.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity for at most `polls` polls; false
// on time-out.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* bar, uint32_t parity, uint32_t polls) {
  for (uint32_t i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Bounded wait of the pipelines (kTmaSpinLimit polls); false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  return mbar_wait_polls(bar, parity, kTmaSpinLimit);
}

__device__ __forceinline__ void report_timeout(int* err, uint64_t* bar, uint32_t parity) {
  if (err) atomicExch(err, kErrTmaTimeout);
  mbar_wait_bounded(bar, parity);  // let copies already in flight land (bounded)
}

}  // namespace su3s
