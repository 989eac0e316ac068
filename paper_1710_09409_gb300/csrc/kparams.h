// Plain-data kernel parameters shared by host planning code and kernels.
#pragma once

#include <cuda.h>   // CUtensorMap (type only)
#include <stdint.h>

namespace su3s {

enum Prec { P_F64 = 0, P_F32 = 1, P_BF16 = 2, P_F16 = 3, P_F64_C12 = 4, P_F32_C12 = 5 };
enum Kind { K_MATRIX = 0, K_VECTOR = 1, K_REAL = 2 };
enum MathId { MATH_F64 = 1, MATH_DF = 2, MATH_F32 = 3, MATH_FX = 4 };

constexpr int kMaxLeaves = 6;
constexpr int kMaxScalars = 4;

// Addressing of one field: element (site s, link mu, component c) is at
//   (s >> logB) * s_blk + mu * s_mu + c * s_c + (s & mask)
// in units of one stored complex (one real for real fields).
struct FieldDesc {
  void* ptr;
  int64_t s_blk;
  int64_t s_mu;
  int64_t s_c;
  int32_t logB;
  uint32_t mask;
  // the same addressing in rows of s_c elements (the rows of the field's
  // 2-D tensor map): component 0 of (s, mu) starts row
  //   (s >> logB) * row_blk + mu * row_mu, at column s & mask
  int32_t row_blk;
  int32_t row_mu;
};

struct KParams {
  // 2-D tensor maps of the leaves (FP64 matrix and vector fields whose
  // 32-site tiles are rows of a 2-D tensor): one tile of all components of an
  // object is one tensor copy.  Valid where the staged kernels run.
  CUtensorMap tm[kMaxLeaves];
  FieldDesc leaf[kMaxLeaves];
  FieldDesc dst;
  double sc[kMaxScalars];   // real factors of scale nodes, in tree order
  float sch[kMaxScalars];   // sc split into FP32 pairs (pair arithmetic)
  float scl[kMaxScalars];
  int64_t nvec;             // site vectors per link (= Vpad / sites per vector)
  int32_t nmu;
  uint32_t gscal;           // range guard: largest high word (sign cleared) of the real factors
  uint32_t ghi;             // range guard bound of the interpreter's program (guard_hi)
  int* err;                 // device error word (bounded waits that gave up), may be null
};

// Adjoint kernels: leaf fields are read, grad_out is read, leaf gradients
// written (ptr == nullptr: skipped).
struct GParams {
  KParams k;                  // leaves, scalars, sizes (k.dst unused)
  CUtensorMap tm_gout;        // tensor map of dL/dZ
  FieldDesc gout;             // dL/dZ
  FieldDesc gleaf[kMaxLeaves];
};

}  // namespace su3s
