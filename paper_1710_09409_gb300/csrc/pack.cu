// Conversion between the canonical AoS FP64 array and a field's device layout
// and storage precision (the scalar/vector data layouts of Sec. 4-5: the
// canonical array is the naive AoS order, the field is the coalesced one).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dev_convert.cuh"
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

// canonical complex index q = (s*nmu + mu)*nc_canon + c; components c >= nc_store skipped
template <int PREC>
__global__ void k_pack(FieldDesc d, const double* __restrict__ canon, int64_t V, int nmu,
                       int nc_canon, int nc_store, int is_real) {
  const int64_t n = V * nmu * nc_canon;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int c = (int)(q % nc_canon);
    const int64_t m = q / nc_canon;
    const int mu = (int)(m % nmu);
    const int64_t s = m / nmu;
    if (c >= nc_store) continue;
    const int64_t e = fbase(d, s, mu) + c * d.s_c;
    if (is_real) reinterpret_cast<double*>(d.ptr)[e] = canon[q];
    else put_complex<PREC>(d.ptr, e, canon[2 * q], canon[2 * q + 1]);
  }
}

template <int PREC>
__global__ void k_zero_pad(FieldDesc d, int64_t V, int64_t Vpad, int nmu, int nc, int is_real) {
  const int64_t np = (Vpad - V) * nmu * nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += stride) {
    const int c = (int)(q % nc);
    const int64_t m = q / nc;
    const int mu = (int)(m % nmu);
    const int64_t s = V + m / nmu;
    const int64_t e = fbase(d, s, mu) + c * d.s_c;
    if (is_real) reinterpret_cast<double*>(d.ptr)[e] = 0.0;
    else put_complex<PREC>(d.ptr, e, 0.0, 0.0);
  }
}

template <int PREC>
__global__ void k_unpack(FieldDesc d, double* __restrict__ canon, int64_t V, int nmu, int nc,
                         int is_real) {
  const int64_t n = V * nmu * nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int c = (int)(q % nc);
    const int64_t m = q / nc;
    const int mu = (int)(m % nmu);
    const int64_t s = m / nmu;
    const int64_t e = fbase(d, s, mu) + c * d.s_c;
    if (is_real) {
      canon[q] = reinterpret_cast<const double*>(d.ptr)[e];
    } else {
      double2 v = get_complex<PREC>(d.ptr, e);
      canon[2 * q] = v.x;
      canon[2 * q + 1] = v.y;
    }
  }
}

// Two-row storage: one thread per matrix, row 2 rebuilt in FP64.
template <int PREC>
__global__ void k_unpack_c12(FieldDesc d, double* __restrict__ canon, int64_t V, int nmu) {
  const int64_t n = V * nmu;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += stride) {
    const int mu = (int)(m % nmu);
    const int64_t s = m / nmu;
    const int64_t b = fbase(d, s, mu);
    double u[18];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double2 v = get_complex<PREC>(d.ptr, b + c * d.s_c);
      u[2 * c] = v.x;
      u[2 * c + 1] = v.y;
    }
    rebuild_row2<MathF64>(u);
#pragma unroll
    for (int r = 0; r < 18; ++r) canon[18 * m + r] = u[r];
  }
}

// Stored-format transfer.  The compact array is site-major like the canonical
// one, but holds per (site, link) only the ncomp stored elements (two rows of a
// C12 matrix), each as the field stores it (T = one element's bytes).  Element
// q = ((s*nmu + mu)*ncomp + c); elements past V*nmu*ncomp are the pad sites,
// which the put kernel zeroes.
template <typename T>
__global__ void k_put_stored(FieldDesc d, const T* __restrict__ src, int64_t V, int64_t Vpad, int nmu,
                             int nc) {
  const int64_t n = V * nmu * nc, np = Vpad * nmu * nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += stride) {
    const int c = (int)(q % nc);
    const int64_t m = q / nc;
    const int mu = (int)(m % nmu);
    const int64_t s = m / nmu;
    reinterpret_cast<T*>(d.ptr)[fbase(d, s, mu) + c * d.s_c] = q < n ? src[q] : T{};
  }
}

template <typename T>
__global__ void k_get_stored(FieldDesc d, T* __restrict__ dst, int64_t V, int nmu, int nc) {
  const int64_t n = V * nmu * nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int c = (int)(q % nc);
    const int64_t m = q / nc;
    const int mu = (int)(m % nmu);
    const int64_t s = m / nmu;
    dst[q] = reinterpret_cast<const T*>(d.ptr)[fbase(d, s, mu) + c * d.s_c];
  }
}

static dim3 grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  int64_t cap = (int64_t)sm_count() * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return dim3((unsigned)b);
}

template <int PREC>
static cudaError_t pack_t(const su3s_field* f, const double* canon, cudaStream_t st) {
  const int is_real = f->kind == SU3S_REAL;
  const int ncc = f->kind == SU3S_MATRIX ? 9 : f->kind == SU3S_VECTOR ? 3 : 1;
  const int64_t n = f->V * f->nmu * ncc;
  if (n > 0) k_pack<PREC><<<grid_for(n), 256, 0, st>>>(f->desc, canon, f->V, f->nmu, ncc, f->ncomp, is_real);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t np = (f->Vpad - f->V) * f->nmu * f->ncomp;
  if (np > 0)
    k_zero_pad<PREC><<<grid_for(np), 256, 0, st>>>(f->desc, f->V, f->Vpad, f->nmu, f->ncomp, is_real);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t unpack_t(const su3s_field* f, double* canon, cudaStream_t st) {
  const int is_real = f->kind == SU3S_REAL;
  if (PREC == P_F64_C12 || PREC == P_F32_C12) {
    const int64_t n = f->V * f->nmu;
    if (n > 0) k_unpack_c12<PREC><<<grid_for(n), 256, 0, st>>>(f->desc, canon, f->V, f->nmu);
  } else {
    const int64_t n = f->V * f->nmu * f->ncomp;
    if (n > 0) k_unpack<PREC><<<grid_for(n), 256, 0, st>>>(f->desc, canon, f->V, f->nmu, f->ncomp, is_real);
  }
  return cudaGetLastError();
}

cudaError_t launch_pack(const su3s_field* f, const double* canon, cudaStream_t st) {
  switch (f->prec) {
    case SU3S_F64: return pack_t<P_F64>(f, canon, st);
    case SU3S_F32: return pack_t<P_F32>(f, canon, st);
    case SU3S_BF16: return pack_t<P_BF16>(f, canon, st);
    case SU3S_F16: return pack_t<P_F16>(f, canon, st);
    case SU3S_F64_C12: return pack_t<P_F64_C12>(f, canon, st);
    default: return pack_t<P_F32_C12>(f, canon, st);
  }
}

cudaError_t launch_unpack(const su3s_field* f, double* canon, cudaStream_t st) {
  switch (f->prec) {
    case SU3S_F64: return unpack_t<P_F64>(f, canon, st);
    case SU3S_F32: return unpack_t<P_F32>(f, canon, st);
    case SU3S_BF16: return unpack_t<P_BF16>(f, canon, st);
    case SU3S_F16: return unpack_t<P_F16>(f, canon, st);
    case SU3S_F64_C12: return unpack_t<P_F64_C12>(f, canon, st);
    default: return unpack_t<P_F32_C12>(f, canon, st);
  }
}

template <typename T>
static cudaError_t put_stored_t(const su3s_field* f, const void* src, cudaStream_t st) {
  const int64_t np = f->Vpad * f->nmu * f->ncomp;
  if (np > 0)
    k_put_stored<T><<<grid_for(np), 256, 0, st>>>(f->desc, (const T*)src, f->V, f->Vpad, f->nmu, f->ncomp);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t get_stored_t(const su3s_field* f, void* dst, cudaStream_t st) {
  const int64_t n = f->V * f->nmu * f->ncomp;
  if (n > 0) k_get_stored<T><<<grid_for(n), 256, 0, st>>>(f->desc, (T*)dst, f->V, f->nmu, f->ncomp);
  return cudaGetLastError();
}

cudaError_t launch_put_stored(const su3s_field* f, const void* src, cudaStream_t st) {
  switch (f->elem_bytes) {
    case 16: return put_stored_t<uint4>(f, src, st);
    case 8: return put_stored_t<uint2>(f, src, st);
    default: return put_stored_t<uint32_t>(f, src, st);
  }
}

cudaError_t launch_get_stored(const su3s_field* f, void* dst, cudaStream_t st) {
  switch (f->elem_bytes) {
    case 16: return get_stored_t<uint4>(f, dst, st);
    case 8: return get_stored_t<uint2>(f, dst, st);
    default: return get_stored_t<uint32_t>(f, dst, st);
  }
}

}  // namespace su3s
