// Whole-field reduction (the loss sum_x Re tr(X^dagger Y)) and projection of
// matrix fields back to SU(3).
#include <math.h>

#include "dev_convert.cuh"
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

constexpr int kRedThreads = 256;

// Fixed-order block reduction of per-thread sums into partial[blockIdx.x].
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sh[0];
}

// sum over real sites s < V, links and components of x*y (FP64 storage)
__global__ void __launch_bounds__(kRedThreads)
    k_redot_partial(FieldDesc x, FieldDesc y, int64_t V, int nmu, int nreal, int is_real,
                    double* __restrict__ partial) {
  const int64_t n = V * nmu;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int mu = (int)(q / V);
    const int64_t s = q - (int64_t)mu * V;
    const int64_t bx = fbase(x, s, mu), by = fbase(y, s, mu);
    if (is_real) {
      acc = fma(reinterpret_cast<const double*>(x.ptr)[bx], reinterpret_cast<const double*>(y.ptr)[by], acc);
    } else {
      for (int c = 0; c < nreal / 2; ++c) {
        const double2 a = reinterpret_cast<const double2*>(x.ptr)[bx + c * x.s_c];
        const double2 b = reinterpret_cast<const double2*>(y.ptr)[by + c * y.s_c];
        acc = fma(a.x, b.x, acc);
        acc = fma(a.y, b.y, acc);
      }
    }
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads)
    k_redot_final(const double* __restrict__ partial, int n, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) *out = t;
}

int redot_blocks() { return 2 * sm_count(); }

cudaError_t launch_redot(const su3s_field* x, const su3s_field* y, double* out, double* partial,
                         int nblocks, cudaStream_t st) {
  const int nreal = x->kind == SU3S_MATRIX ? 18 : x->kind == SU3S_VECTOR ? 6 : 1;
  k_redot_partial<<<nblocks, kRedThreads, 0, st>>>(x->desc, y->desc, x->V, x->nmu, nreal,
                                                   x->kind == SU3S_REAL, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_redot_final<<<1, kRedThreads, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

int check_redot(const su3s_field* x, const su3s_field* y, const double* out) {
  if (!x || !y || !out) return fail(SU3S_EINVAL, "null argument");
  if (x->kind != y->kind) return fail(SU3S_ETYPE, "fields of different kinds");
  if (x->prec != SU3S_F64 || y->prec != SU3S_F64)
    return fail(SU3S_EUNSUPPORTED, "reduction needs FP64 storage");
  return check_same_shape(x, y, true);
}

// ------------------------------------------------------------ reunitarise
template <int PREC>
__global__ void __launch_bounds__(256) k_reunit(FieldDesc src, FieldDesc dst, int64_t V, int nmu) {
  const int64_t n = V * nmu;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const int mu = (int)(q / V);
    const int64_t s = q - (int64_t)mu * V;
    const int64_t bs = fbase(src, s, mu), bd = fbase(dst, s, mu);
    double r[18];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      double2 v = get_complex<PREC>(src.ptr, bs + c * src.s_c);
      r[2 * c] = v.x;
      r[2 * c + 1] = v.y;
    }
    // Gram-Schmidt over rows, two projection sweeps
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int rep = 0; rep < 2; ++rep)
#pragma unroll
        for (int p = 0; p < i; ++p) {
          double cr = 0.0, ci = 0.0;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double pr = r[6 * p + 2 * j], pi = r[6 * p + 2 * j + 1];
            const double xr = r[6 * i + 2 * j], xi = r[6 * i + 2 * j + 1];
            cr += pr * xr + pi * xi;
            ci += pr * xi - pi * xr;
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double pr = r[6 * p + 2 * j], pi = r[6 * p + 2 * j + 1];
            r[6 * i + 2 * j] -= cr * pr - ci * pi;
            r[6 * i + 2 * j + 1] -= cr * pi + ci * pr;
          }
        }
      double nn = 0.0;
#pragma unroll
      for (int j = 0; j < 6; ++j) nn += r[6 * i + j] * r[6 * i + j];
      const double inv = rsqrt(nn);
#pragma unroll
      for (int j = 0; j < 6; ++j) r[6 * i + j] *= inv;
    }
    double dr = 0.0, di = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int a = (j + 1) % 3, b = (j + 2) % 3;
      const double xr = r[6 + 2 * a] * r[12 + 2 * b] - r[6 + 2 * a + 1] * r[12 + 2 * b + 1] -
                        (r[6 + 2 * b] * r[12 + 2 * a] - r[6 + 2 * b + 1] * r[12 + 2 * a + 1]);
      const double xi = r[6 + 2 * a] * r[12 + 2 * b + 1] + r[6 + 2 * a + 1] * r[12 + 2 * b] -
                        (r[6 + 2 * b] * r[12 + 2 * a + 1] + r[6 + 2 * b + 1] * r[12 + 2 * a]);
      dr += r[2 * j] * xr - r[2 * j + 1] * xi;
      di += r[2 * j] * xi + r[2 * j + 1] * xr;
    }
    const double phi = atan2(di, dr);
    double sn, cs;
    sincos(-phi / 3.0, &sn, &cs);
#pragma unroll
    for (int c = 0; c < 9; ++c)
      put_complex<PREC>(dst.ptr, bd + c * dst.s_c, cs * r[2 * c] - sn * r[2 * c + 1],
                        cs * r[2 * c + 1] + sn * r[2 * c]);
  }
}

template <int PREC>
static cudaError_t reunit_t(const su3s_field* src, su3s_field* dst, cudaStream_t st) {
  const int64_t n = src->V * src->nmu;
  int64_t nb = (n + 255) / 256;
  if (nb > (int64_t)sm_count() * 16) nb = (int64_t)sm_count() * 16;
  if (nb < 1) nb = 1;
  k_reunit<PREC><<<(unsigned)nb, 256, 0, st>>>(src->desc, dst->desc, src->V, src->nmu);
  return cudaGetLastError();
}

}  // namespace su3s

using namespace su3s;

SU3S_EXPORT int su3s_field_redot(const su3s_field* x, const su3s_field* y, double* dev_out,
                                 void* stream) {
  int rc = check_redot(x, y, dev_out);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = redot_blocks();
  void* partial = nullptr;
  cudaError_t e = scratch_alloc(&partial, nb * sizeof(double), st);
  if (e != cudaSuccess) return fail(SU3S_ENOMEM, "reduction scratch: %s", cudaGetErrorString(e));
  e = launch_redot(x, y, dev_out, (double*)partial, nb, st);
  cudaError_t e2 = scratch_free(partial, st);
  if (e != cudaSuccess) return cuda_fail(e, "reduction kernels");
  if (e2 != cudaSuccess) return cuda_fail(e2, "reduction scratch release");
  return SU3S_OK;
}

SU3S_EXPORT int su3s_reunitarize(su3s_field* dst, const su3s_field* src, void* stream) {
  if (!dst || !src) return fail(SU3S_EINVAL, "null argument");
  if (src->kind != SU3S_MATRIX || dst->kind != SU3S_MATRIX)
    return fail(SU3S_ETYPE, "projection to SU(3) needs matrix fields");
  int rc = check_same_shape(src, dst, true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (src->prec) {
    case SU3S_F64: e = reunit_t<P_F64>(src, dst, st); break;
    case SU3S_F32: e = reunit_t<P_F32>(src, dst, st); break;
    case SU3S_BF16: e = reunit_t<P_BF16>(src, dst, st); break;
    case SU3S_F16: e = reunit_t<P_F16>(src, dst, st); break;
    default: return fail(SU3S_EUNSUPPORTED, "two-row storage is special unitary by construction");
  }
  if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
  return SU3S_OK;
}
