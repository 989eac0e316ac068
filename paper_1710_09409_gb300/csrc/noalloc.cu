// Download without any device allocation: the unpack kernel writes into a
// fixed staging array that lives in this module's device memory instead of
// a buffer allocated per call.
//
// For callers that cannot allocate device memory when they download a field:
// a framework whose caching allocator already holds the device's memory (a new
// allocation by this library can then fail although the framework has free
// space), or code that must not pay the latency or the implicit
// synchronisation that allocating and freeing device memory can bring.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

// 16 MiB of staging, held by every GPU on which this library is used until
// the process exits.  Every call shares it; it keeps the last call's contents.
constexpr size_t kStaticStageDoubles = (size_t)2 << 20;
static __device__ __align__(256) double g_static_stage[kStaticStageDoubles];

// Device address of the staging array on the current device, looked up once
// per device (with that device current) and cached.  The first lookup on a
// device loads this file's module there, which places the array in device
// memory; su3s_field_wrap does it (field creation may allocate), so a
// download of a wrapped field finds the address cached.  The cache is not
// invalidated: a device reset while the library is loaded is not supported.
static int static_stage_ptr(double** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static double* ptrs[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "current device");
  if (dev < 0 || dev >= kMaxDevices) return fail(SU3S_EUNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_stage);
    if (e != cudaSuccess) return cuda_fail(e, "address of the static staging array");
    ptrs[dev] = (double*)p;
  }
  *out = ptrs[dev];
  return SU3S_OK;
}

int prepare_static_stage() {
  double* p = nullptr;
  return static_stage_ptr(&p);
}

}  // namespace su3s

using namespace su3s;

SU3S_EXPORT int su3s_field_download_static(const su3s_field* f, double* host_canonical,
                                           size_t n_doubles, void* stream) {
  if (!f || !host_canonical) return fail(SU3S_EINVAL, "null argument");
  const int w = f->kind == SU3S_MATRIX ? 18 : f->kind == SU3S_VECTOR ? 6 : 1;
  const size_t need = (size_t)f->V * f->nmu * w;
  if (n_doubles != need)
    return fail(SU3S_ESHAPE, "host array has %zu doubles, the field holds %zu", n_doubles, need);
  if (need > kStaticStageDoubles)
    return fail(SU3S_ESHAPE,
                "field needs %zu doubles of staging; the static staging area holds %zu "
                "(16 MiB): use su3s_field_download for larger fields",
                need, kStaticStageDoubles);
  double* stage = nullptr;
  int rc = static_stage_ptr(&stage);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_unpack(f, stage, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_canonical, stage, need * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "static-staging download");
  return SU3S_OK;
}
