/* A plain C99 client of the su3s C ABI, built by tests/test_c_client.py with
 * -std=c99 -Wall -Wextra -Werror against include/su3s.h and linked to the
 * library.  It uses only the host side of the ABI (no kernel is launched):
 * lattice creation, field sizes, wrapping a device address that is never
 * dereferenced, building a*b + c*d, its canonical signature and the catalogue
 * entry it maps to, and the error path.  Prints "ok" and exits 0 on success. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "su3s.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (call);                                                        \
    if (rc_ != SU3S_OK) {                                                    \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, su3s_last_error()); \
      return 1;                                                              \
    }                                                                        \
  } while (0)

int main(void) {
  su3s_lattice* lat = NULL;
  CHECK(su3s_lattice_create(4, 4, 4, 6, &lat));
  int64_t vol = 0;
  CHECK(su3s_lattice_volume(lat, &vol));
  if (vol != 384) return 2;

  size_t bytes = 0;
  CHECK(su3s_field_bytes(lat, SU3S_MATRIX, 1, SU3S_F64, SU3S_SOA, 0, &bytes));
  if (bytes != (size_t)384 * 9 * 16) return 3;

  /* four fields at distinct 16-byte aligned addresses, never dereferenced */
  su3s_field* f[4];
  for (int i = 0; i < 4; ++i) {
    void* addr = (void*)(uintptr_t)((1ull << 40) + (uint64_t)i * (1ull << 24));
    CHECK(su3s_field_wrap(lat, SU3S_MATRIX, 1, SU3S_F64, SU3S_SOA, 0, addr, bytes, &f[i]));
  }
  size_t stored = 0;
  CHECK(su3s_field_stored_bytes(f[0], &stored));
  if (stored != (size_t)384 * 9 * 16) return 4;

  su3s_expr *a, *b, *c, *d, *ab, *cd, *e;
  CHECK(su3s_expr_leaf(f[0], &a));
  CHECK(su3s_expr_leaf(f[1], &b));
  CHECK(su3s_expr_leaf(f[2], &c));
  CHECK(su3s_expr_leaf(f[3], &d));
  CHECK(su3s_expr_mul(a, b, &ab));
  CHECK(su3s_expr_mul(c, d, &cd));
  CHECK(su3s_expr_add(ab, cd, &e));
  /* children may be freed once the parent holds them */
  CHECK(su3s_expr_free(ab));
  CHECK(su3s_expr_free(cd));

  char sig[256];
  CHECK(su3s_expr_signature(e, sig, sizeof sig));
  if (strcmp(sig, "add(mul(M0,M1),mul(M2,M3))") != 0) return 5;
  int n = 0;
  CHECK(su3s_expr_num_leaves(e, &n));
  if (n != 4) return 6;

  char* cat = (char*)malloc(1 << 16);
  if (!cat) return 7;
  CHECK(su3s_catalogue(cat, 1 << 16));
  if (!strstr(cat, "eval add(mul(M0,M1),mul(M2,M3)) f64 df32")) return 8;
  free(cat);

  /* the error path: a vector times a matrix is ill-typed */
  su3s_field* fv = NULL;
  size_t vbytes = 0;
  CHECK(su3s_field_bytes(lat, SU3S_VECTOR, 1, SU3S_F64, SU3S_SOA, 0, &vbytes));
  CHECK(su3s_field_wrap(lat, SU3S_VECTOR, 1, SU3S_F64, SU3S_SOA, 0,
                        (void*)(uintptr_t)(1ull << 41), vbytes, &fv));
  su3s_expr *v = NULL, *bad = NULL;
  CHECK(su3s_expr_leaf(fv, &v));
  if (su3s_expr_mul(v, a, &bad) != SU3S_ETYPE || bad != NULL) return 9;
  if (strlen(su3s_last_error()) == 0) return 10;

  CHECK(su3s_expr_free(v));
  CHECK(su3s_expr_free(e));
  CHECK(su3s_expr_free(a));
  CHECK(su3s_expr_free(b));
  CHECK(su3s_expr_free(c));
  CHECK(su3s_expr_free(d));
  CHECK(su3s_field_destroy(fv));
  for (int i = 0; i < 4; ++i) CHECK(su3s_field_destroy(f[i]));
  CHECK(su3s_lattice_destroy(lat));
  printf("ok %d\n", su3s_version());
  return 0;
}
