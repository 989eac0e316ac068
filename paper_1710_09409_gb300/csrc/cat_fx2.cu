// Catalogue of compiled trees, FP64 storage, shared-exponent fixed-point arithmetic:
// fused multi-term trees.
#include "dev_kernels.cuh"
#include "internal.h"

namespace su3s {

void register_cat_fx2() {
  using namespace cat;
  constexpr int P = P_F64;
  using M = MathFX;
  const int m = MATH_FX;
  reg_eval<E1, M, P>(m);
  reg_eval<E1Sub, M, P>(m);
  reg_eval<E1Lin, M, P>(m);
  reg_eval<E2, M, P>(m);
  reg_eval<MMM, M, P>(m);
  reg_eval<E3, M, P>(m);
  reg_eval<Comm, M, P>(m);
}

}  // namespace su3s
