/* A C99 program that uses the su3s C ABI end to end on the GPU, with no Python
 * and no framework: device memory from cudaMalloc, seeded SU(3) inputs from
 * the synth library, upload, one-pass evaluation of z = a*b and of its reverse
 * mode, download, and a check against the CPU oracle's C library.  Built and
 * run by tests/test_c_client.py (GPU test).  Prints "ok <max error>" and
 * exits 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "su3s.h"

/* the seeded input generator and the oracle (their own C libraries) */
int synth_fill(int kind, uint64_t seed, uint32_t field, int64_t first, int64_t count, double* out,
               int nthreads);
void oracle_mm(const double* x, const double* y, double* z, int64_t n);

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != SU3S_OK) {                                                    \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, su3s_last_error()); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

static double max_abs_diff(const double* x, const double* y, size_t n) {
  double m = 0.0;
  for (size_t i = 0; i < n; ++i) {
    const double d = fabs(x[i] - y[i]);
    if (d > m) m = d;
  }
  return m;
}

int main(void) {
  const int L[4] = {8, 8, 8, 9};
  su3s_lattice* lat = NULL;
  CHECK(su3s_lattice_create(L[0], L[1], L[2], L[3], &lat));
  int64_t V = 0;
  CHECK(su3s_lattice_volume(lat, &V));
  const size_t nd = (size_t)V * 18;

  size_t bytes = 0;
  CHECK(su3s_field_bytes(lat, SU3S_MATRIX, 1, SU3S_F64, SU3S_SOA, 0, &bytes));
  void* mem[5];
  su3s_field* f[5]; /* a, b, z, dA, dB (W reuses z's memory after the forward check) */
  for (int i = 0; i < 5; ++i) {
    if (cudaMalloc(&mem[i], bytes) != cudaSuccess) return 2;
    CHECK(su3s_field_wrap(lat, SU3S_MATRIX, 1, SU3S_F64, SU3S_SOA, 0, mem[i], bytes, &f[i]));
  }

  double* ha = (double*)malloc(nd * sizeof(double));
  double* hb = (double*)malloc(nd * sizeof(double));
  double* hz = (double*)malloc(nd * sizeof(double));
  double* ref = (double*)malloc(nd * sizeof(double));
  if (!ha || !hb || !hz || !ref) return 3;
  const uint64_t seed = 1710094090u;
  if (synth_fill(0, seed, 0, 0, V, ha, 1) || synth_fill(0, seed, 1, 0, V, hb, 1)) return 4;
  CHECK(su3s_field_upload(f[0], ha, nd, NULL));
  CHECK(su3s_field_upload(f[1], hb, nd, NULL));

  /* forward: z = a*b */
  su3s_expr *a, *b, *ab;
  CHECK(su3s_expr_leaf(f[0], &a));
  CHECK(su3s_expr_leaf(f[1], &b));
  CHECK(su3s_expr_mul(a, b, &ab));
  CHECK(su3s_eval(f[2], ab, NULL));
  CHECK(su3s_field_download(f[2], hz, nd, NULL));
  if (cudaDeviceSynchronize() != cudaSuccess) return 5;
  oracle_mm(ha, hb, ref, V);
  const double err = max_abs_diff(hz, ref, nd);
  if (!(err < 1e-13)) {
    fprintf(stderr, "z = a*b differs from the oracle by %g\n", err);
    return 6;
  }

  /* reverse mode for dL/dz = W = a (an SU(3) field): dA = W b^dagger = a b^dagger,
     dB = a^dagger W = a^dagger a = I */
  su3s_field* grads[2] = {f[3], f[4]};
  CHECK(su3s_eval_adjoint(ab, f[0], grads, 2, SU3S_MATH_DEFAULT, NULL));
  CHECK(su3s_field_download(f[4], hz, nd, NULL));
  if (cudaDeviceSynchronize() != cudaSuccess) return 7;
  double gerr = 0.0;
  for (int64_t s = 0; s < V; ++s)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double* e = hz + 18 * s + 2 * (3 * i + j);
        const double dre = fabs(e[0] - (i == j ? 1.0 : 0.0)), dim = fabs(e[1]);
        if (dre > gerr) gerr = dre;
        if (dim > gerr) gerr = dim;
      }
  if (!(gerr < 1e-13)) {
    fprintf(stderr, "dB = a^dagger a differs from the identity by %g\n", gerr);
    return 8;
  }
  int code = -1;
  CHECK(su3s_device_error(&code, NULL));
  if (code != 0) return 9;

  CHECK(su3s_expr_free(ab));
  CHECK(su3s_expr_free(a));
  CHECK(su3s_expr_free(b));
  for (int i = 0; i < 5; ++i) {
    CHECK(su3s_field_destroy(f[i]));
    cudaFree(mem[i]);
  }
  CHECK(su3s_lattice_destroy(lat));
  free(ha);
  free(hb);
  free(hz);
  free(ref);
  printf("ok %.3g %.3g\n", err, gerr);
  return 0;
}
